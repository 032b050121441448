// summarize.cu -- stage 1: one streaming pass over the input that writes
// per-64-byte-block summaries for the chain stage.
//
//   RAM / AE : block maximum and the offset of its first occurrence
//              (Extreme Byte Search of Section 3.1 applied to every block at
//              once). AE-Min uses the complemented bytes.
//   MAXP     : the offset of the block's target, if any: a byte strictly
//              greater than every byte within distance w on both sides
//              (Section 2.1, MAXP). With w >= 63 a whole block lies within
//              any target's windows, so a target is the block's unique
//              maximum; it is then checked against the neighbouring blocks'
//              maxima, and against raw bytes only for the two partial blocks
//              at the window ends.
//
// Data movement: persistent CTAs stream 16 KiB tiles from HBM into a ring of
// shared-memory stages with 1-D bulk copies (cp.async.bulk + mbarrier
// complete_tx); all threads then read the tile with conflict-free 16-byte
// shared loads. The kernel is bound by HBM bandwidth: it reads each input
// byte once and writes 2 bytes (1 for MAXP) per 64 input bytes.
#include "cdc_device.cuh"
#include "cdc_launch.h"

namespace cdc {

constexpr int S1_THREADS = 256;
constexpr int S1_TILE = 16384;
constexpr int S1_STAGES = 4;

// Bytes of a 16-byte chunk at physical position `pos` outside [lo, hi) -> 0.
__device__ __forceinline__ void mask16(uint32_t w[4], uint64_t pos, uint64_t lo, uint64_t hi) {
    if (pos >= lo && pos + 16 <= hi) return;
#pragma unroll
    for (int k = 0; k < 4; k++) w[k] = clip_word(w[k], (pos >> 2) + k, lo, hi);
}

__device__ __forceinline__ void reset_ctrl(Ctrl* c) {
    c->ticket = 0;
    c->total = 0;
    c->epoch = c->epoch + 1;
}

__global__ void k_reset(Ctrl* ctrl) {
    if (threadIdx.x == 0 && blockIdx.x == 0) reset_ctrl(ctrl);
}

// max and first argmax of one 16-byte chunk, as a key (max << 8) | (63 - pos)
__device__ __forceinline__ uint32_t chunk_key(const uint32_t w[4], uint32_t q) {
    uint32_t m = vmax4(vmax4(w[0], w[1]), vmax4(w[2], w[3]));
    uint32_t M = hmax4(m), Mx = M * 0x01010101u;
    uint32_t e0 = vcmpeq4(w[0], Mx), e1 = vcmpeq4(w[1], Mx), e2 = vcmpeq4(w[2], Mx), e3 = vcmpeq4(w[3], Mx);
    uint32_t idx = e0 ? ((ffs32(e0) - 1) >> 3)
                      : e1 ? 4 + ((ffs32(e1) - 1) >> 3) : e2 ? 8 + ((ffs32(e2) - 1) >> 3) : 12 + ((ffs32(e3) - 1) >> 3);
    return (M << 8) | (63u - (16u * q + idx));
}

// last argmax key of one chunk for the block maximum M: (M << 8) | pos, or 0
// when the chunk holds no byte equal to M
__device__ __forceinline__ uint32_t chunk_key_last(const uint32_t w[4], uint32_t q, uint32_t M) {
    uint32_t Mx = M * 0x01010101u;
    uint32_t e0 = vcmpeq4(w[0], Mx), e1 = vcmpeq4(w[1], Mx), e2 = vcmpeq4(w[2], Mx), e3 = vcmpeq4(w[3], Mx);
    if ((e0 | e1 | e2 | e3) == 0) return 0;
    uint32_t idx = e3 ? 12 + ((31 - __clz(e3)) >> 3)
                      : e2 ? 8 + ((31 - __clz(e2)) >> 3) : e1 ? 4 + ((31 - __clz(e1)) >> 3) : ((31 - __clz(e0)) >> 3);
    return (M << 8) | (16u * q + idx);
}

// issue the copy of bytes [r0, r1) (physical positions) into the stage buffer
// `dst`, whose first byte stands for position r0; clipped to [glo, ghi).
__device__ __forceinline__ void issue_tile(const uint8_t* base, uint64_t glo, uint64_t ghi, uint64_t r0,
                                           uint64_t r1, uint8_t* dst, uint64_t* bar) {
    uint64_t c0 = r0 > glo ? r0 : glo, c1 = r1 < ghi ? r1 : ghi;
    if (c1 > c0) {
        uint32_t bytes = (uint32_t)(c1 - c0);
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(dst + (c0 - r0), base + c0, bytes, bar);
    } else {
        mbar_arrive(bar);
    }
}

// ---- RAM / AE summaries ------------------------------------------------------

template <bool INV>
__global__ void __launch_bounds__(S1_THREADS) k_summary_max(SumLaunch a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* buf = smem;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S1_STAGES * S1_TILE);
    __shared__ unsigned int supmax[S1_STAGES][S1_TILE / 4096];
    const int tid = threadIdx.x;
    if (blockIdx.x == 0 && tid == 0) reset_ctrl(a.ctrl);
    const uint64_t ntiles = (a.nblk * 64 + S1_TILE - 1) / S1_TILE;
    if (tid == 0) {
        for (int s = 0; s < S1_STAGES; s++) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    if (tid < S1_STAGES * (S1_TILE / 4096)) (&supmax[0][0])[tid] = 0;
    __syncthreads();
    const uint64_t g = gridDim.x;
    if (tid == 0) {
        for (int s = 0; s < S1_STAGES; s++) {
            uint64_t t = blockIdx.x + s * g;
            if (t < ntiles)
                issue_tile(a.base, a.glo, a.ghi, t * S1_TILE, t * S1_TILE + S1_TILE, buf + s * S1_TILE, &bar[s]);
        }
    }
    const uint32_t inv = INV ? 0xFFFFFFFFu : 0u;
    uint32_t i = 0;
    for (uint64_t t = blockIdx.x; t < ntiles; t += g, i++) {
        const int s = i % S1_STAGES;
        const uint32_t par = (i / S1_STAGES) & 1u;
        if (!mbar_wait_bounded(&bar[s], par, a.timeout_ns)) {
            atomicOr(&a.ctrl->err, ERR_TIMEOUT);
            // wait (bounded) for the copies still in flight before leaving
            for (int k = 0; k < S1_STAGES; k++) mbar_wait_bounded(&bar[k], par, a.timeout_ns);
            return;
        }
        const uint8_t* tb = buf + s * S1_TILE;
        const uint64_t T0 = t * S1_TILE;
#pragma unroll
        for (int it = 0; it < S1_TILE / 16 / S1_THREADS; it++) {
            const uint32_t c = it * S1_THREADS + tid;  // 16-byte chunk in tile
            uint4 v = reinterpret_cast<const uint4*>(tb)[c];
            uint32_t w[4] = {v.x ^ inv, v.y ^ inv, v.z ^ inv, v.w ^ inv};
            mask16(w, T0 + 16ull * c, a.lo, a.hi);
            uint32_t key = chunk_key(w, c & 3u);
            key = max(key, __shfl_xor_sync(FULL, key, 1));
            key = max(key, __shfl_xor_sync(FULL, key, 2));
            if ((c & 3u) == 0) {
                uint64_t b = T0 / 64 + (c >> 2);
                if (b < a.nblk) {
                    a.smax[b] = (uint8_t)(key >> 8);
                    a.sarg[b] = (uint8_t)(63u - (key & 0xFFu));
                }
            }
            // each iteration covers one 4 KiB superblock of the tile
            uint32_t wm = __reduce_max_sync(FULL, key >> 8);
            if ((tid & 31) == 0 && wm) atomicMax(&supmax[s][it], wm);
        }
        __syncthreads();  // every thread is done with stage s
        if (tid < S1_TILE / 4096) {
            uint64_t q = T0 / 4096 + tid;
            if (q < a.nsup) a.ssup[q] = (uint8_t)supmax[s][tid];
            supmax[s][tid] = 0;
        }
        if (tid == 0) {
            uint64_t tn = t + S1_STAGES * g;
            if (tn < ntiles)
                issue_tile(a.base, a.glo, a.ghi, tn * S1_TILE, tn * S1_TILE + S1_TILE, buf + s * S1_TILE, &bar[s]);
        }
    }
}

// ---- MAXP targets --------------------------------------------------------------

constexpr int MP_THREADS = 256;
constexpr int MP_TILE_BLOCKS = 256;  // 16 KiB of targets per tile

// Dynamic shared memory: 2 stages of (MP_TILE_BLOCKS + 2*hb) * 64 bytes, then
// per-stage-block max / first / last arrays, then 2 mbarriers.
__global__ void __launch_bounds__(MP_THREADS) k_summary_maxp(SumLaunch a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x;
    const uint32_t hb = a.halo_blocks;
    const uint32_t nb = MP_TILE_BLOCKS + 2 * hb;  // blocks per stage
    const uint32_t sbytes = nb * 64;
    uint8_t* buf = smem;
    uint8_t* bm = smem + 2 * sbytes;
    uint8_t* bf = bm + nb;
    uint8_t* bl = bf + nb;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + ((2 * sbytes + 3 * nb + 15) & ~15u));
    __shared__ unsigned int supcnt[MP_TILE_BLOCKS / 64];
    if (blockIdx.x == 0 && tid == 0) reset_ctrl(a.ctrl);
    const uint64_t ntiles = (a.nblk + MP_TILE_BLOCKS - 1) / MP_TILE_BLOCKS;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if (tid < MP_TILE_BLOCKS / 64) supcnt[tid] = 0;
    __syncthreads();
    const uint64_t g = gridDim.x;
    // stage block 0 stands for global block t * MP_TILE_BLOCKS - hb (negative
    // positions and positions outside [glo, ghi) are not copied)
    auto issue = [&](uint64_t t, int s) {
        int64_t r0 = ((int64_t)(t * MP_TILE_BLOCKS) - (int64_t)hb) * 64, r1 = r0 + (int64_t)sbytes;
        int64_t c0 = r0 > (int64_t)a.glo ? r0 : (int64_t)a.glo;
        int64_t c1 = r1 < (int64_t)a.ghi ? r1 : (int64_t)a.ghi;
        uint8_t* dst = buf + s * sbytes;
        if (c1 > c0) {
            uint32_t bytes = (uint32_t)(c1 - c0);
            mbar_arrive_expect_tx(&bar[s], bytes);
            bulk_g2s(dst + (c0 - r0), a.base + c0, bytes, &bar[s]);
        } else {
            mbar_arrive(&bar[s]);
        }
    };
    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            uint64_t t = blockIdx.x + s * g;
            if (t < ntiles) issue(t, s);
        }
    }
    const uint32_t w = a.w;
    uint32_t i = 0;
    for (uint64_t t = blockIdx.x; t < ntiles; t += g, i++) {
        const int s = i & 1;
        const uint32_t par = (i >> 1) & 1u;
        if (!mbar_wait_bounded(&bar[s], par, a.timeout_ns)) {
            atomicOr(&a.ctrl->err, ERR_TIMEOUT);
            mbar_wait_bounded(&bar[0], par, a.timeout_ns);
            mbar_wait_bounded(&bar[1], par, a.timeout_ns);
            return;
        }
        const uint8_t* tb = buf + s * sbytes;
        const int64_t sb0 = (int64_t)(t * MP_TILE_BLOCKS) - (int64_t)hb;  // global block of stage block 0
        // 1) block max, first and last position of the max, for every stage block
        for (uint32_t cb = 0; cb < nb * 4; cb += MP_THREADS) {
            // every thread takes part in the shuffles; chunks past the stage are zeros
            const uint32_t c = cb + tid;
            const bool act = c < nb * 4;
            uint4 v = act ? reinterpret_cast<const uint4*>(tb)[c] : make_uint4(0, 0, 0, 0);
            uint32_t wd[4] = {v.x, v.y, v.z, v.w};
            int64_t pos = (sb0 + (int64_t)(c >> 2)) * 64 + 16 * (int64_t)(c & 3u);
            if (pos < 0 || (uint64_t)pos < a.lo || (uint64_t)pos + 16 > a.hi) {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (pos < 0) wd[k] = 0;
                    else wd[k] = clip_word(wd[k], ((uint64_t)pos >> 2) + k, a.lo, a.hi);
                }
            }
            uint32_t kf = chunk_key(wd, c & 3u);
            kf = max(kf, __shfl_xor_sync(FULL, kf, 1));
            kf = max(kf, __shfl_xor_sync(FULL, kf, 2));
            uint32_t M = kf >> 8;
            uint32_t kl = chunk_key_last(wd, c & 3u, M);
            kl = max(kl, __shfl_xor_sync(FULL, kl, 1));
            kl = max(kl, __shfl_xor_sync(FULL, kl, 2));
            if (act && (c & 3u) == 0) {
                bm[c >> 2] = (uint8_t)M;
                bf[c >> 2] = (uint8_t)(63u - (kf & 0xFFu));
                bl[c >> 2] = (uint8_t)(kl & 0xFFu);
            }
        }
        __syncthreads();
        // 2) target test, one thread per tile block
        for (uint32_t lb = tid; lb < MP_TILE_BLOCKS; lb += MP_THREADS) {  // one block per thread
            const uint64_t gb = t * MP_TILE_BLOCKS + lb;
            const uint32_t sbi = hb + lb;  // stage index of this block
            const uint32_t v = bm[sbi];
            const uint64_t p = gb * 64 + bf[sbi];
            bool ok = gb < a.nblk && v != 0 && bf[sbi] == bl[sbi] && p >= a.lo + w && p + w < a.hi;
            if (ok) {
                const uint64_t wl = p - w, wr = p + w;  // window [wl, wr]
                const uint64_t kb0 = wl >> 6, kb1 = wr >> 6;
                for (uint64_t kb = kb0; kb <= kb1 && ok; kb++) {
                    if (kb == gb) continue;
                    const uint32_t si = (uint32_t)((int64_t)kb - sb0);
                    if (bm[si] < v) continue;
                    const uint64_t blo = kb * 64, bhi = blo + 63;
                    if (blo >= wl && bhi <= wr) { ok = false; break; }
                    const uint64_t x0 = blo > wl ? blo : wl, x1 = bhi < wr ? bhi : wr;
                    const uint8_t* sp = tb + (size_t)si * 64;
                    for (uint64_t x = x0; x <= x1; x++)
                        if (sp[x - blo] >= v) { ok = false; break; }
                }
            }
            if (gb < a.nblk) a.smax[gb] = ok ? bf[sbi] : (uint8_t)0xFFu;
            // targets per 4 KiB superblock (64 blocks = 2 warps of this loop)
            const uint32_t cntw = __popc(__ballot_sync(FULL, ok));
            if ((tid & 31) == 0 && cntw) atomicAdd(&supcnt[lb >> 6], cntw);
        }
        __syncthreads();
        if (tid < MP_TILE_BLOCKS / 64) {
            uint64_t q = t * (MP_TILE_BLOCKS / 64) + tid;
            if (q < a.nsup) a.ssup[q] = (uint8_t)min(supcnt[tid], 255u);
            supcnt[tid] = 0;
        }
        __syncthreads();
        if (tid == 0) {
            uint64_t tn = t + 2 * g;
            if (tn < ntiles) issue(tn, s);
        }
    }
}

// ---- launchers -----------------------------------------------------------------

int summary_max_smem() { return S1_STAGES * S1_TILE + S1_STAGES * 8; }

int summary_maxp_smem(uint32_t halo_blocks) {
    uint32_t nb = MP_TILE_BLOCKS + 2 * halo_blocks;
    return (int)(((2 * nb * 64 + 3 * nb + 15) & ~15u) + 16);
}

uint32_t maxp_halo_blocks(uint32_t w) { return (w + 63) / 64 + 1; }

cudaError_t launch_summary(const SumLaunch& a, int kind, int grid, cudaStream_t st) {
    if (kind == SUM_MAXP) {
        int sm = summary_maxp_smem(a.halo_blocks);
        cudaError_t e = cudaFuncSetAttribute(k_summary_maxp, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        k_summary_maxp<<<grid, MP_THREADS, sm, st>>>(a);
    } else {
        int sm = summary_max_smem();
        if (kind == SUM_MAX_INV) {
            cudaError_t e = cudaFuncSetAttribute(k_summary_max<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e != cudaSuccess) return e;
            k_summary_max<true><<<grid, S1_THREADS, sm, st>>>(a);
        } else {
            cudaError_t e = cudaFuncSetAttribute(k_summary_max<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e != cudaSuccess) return e;
            k_summary_max<false><<<grid, S1_THREADS, sm, st>>>(a);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_reset(Ctrl* ctrl, cudaStream_t st) {
    k_reset<<<1, 32, 0, st>>>(ctrl);
    return cudaGetLastError();
}

int summary_blocks_per_sm(int kind, uint32_t halo_blocks) {
    int n = 0;
    if (kind == SUM_MAXP) {
        int sm = summary_maxp_smem(halo_blocks);
        cudaFuncSetAttribute(k_summary_maxp, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_summary_maxp, MP_THREADS, sm);
    } else {
        int sm = summary_max_smem();
        cudaFuncSetAttribute(k_summary_max<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_summary_max<false>, S1_THREADS, sm);
    }
    return n > 0 ? n : 1;
}

uint64_t summary_tiles(int kind, uint64_t nblk) {
    return kind == SUM_MAXP ? (nblk + MP_TILE_BLOCKS - 1) / MP_TILE_BLOCKS : (nblk * 64 + S1_TILE - 1) / S1_TILE;
}

}  // namespace cdc
