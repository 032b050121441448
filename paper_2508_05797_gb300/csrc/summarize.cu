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
// Data movement: persistent CTAs stream 16 KiB tiles (MAXP: 32 KiB and a halo
// on each side) from HBM into a ring of shared-memory stages with 1-D bulk
// copies (cp.async.bulk + mbarrier complete_tx); all threads then read the
// tile with conflict-free 16-byte shared loads. The kernel is bound by HBM bandwidth: it reads each input
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

// Maximum and first (LAST = false) or last (LAST = true) position of the
// maximum of one 64-byte block held in shared memory, as the key
// (max << 8) | tag, tag = 255 - position (first) or position (last).
// Bytes go into 16-bit lanes next to their position tag with byte permutes,
// so one native 16x2 max takes two bytes at a time and ties resolve to the
// wanted end. The block's four 16-byte columns are read in the order
// k ^ sw, which spreads a warp's reads over all shared-memory banks.
// Bytes outside [lo, hi) count as 0 (after the complement `inv`).
template <bool LAST>
__device__ __forceinline__ uint32_t block_key(const uint8_t* blk, uint32_t sw, uint32_t inv, bool edge, uint64_t p0,
                                              uint64_t lo, uint64_t hi) {
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t c = (uint32_t)k ^ sw;
        const uint4 v = *reinterpret_cast<const uint4*>(blk + 16 * c);
        uint32_t w[4] = {v.x ^ inv, v.y ^ inv, v.z ^ inv, v.w ^ inv};
        if (edge) mask16(w, p0 + 16 * c, lo, hi);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t base = 16u * c + 4u * (uint32_t)j;  // position of the word's byte 0
            const uint32_t tag = LAST ? 0x03020100u + base * 0x01010101u : 0xFCFDFEFFu - base * 0x01010101u;
            const uint32_t e = __byte_perm(w[j], tag, 0x2604);  // lanes (b0 << 8 | t0), (b2 << 8 | t2)
            const uint32_t o = __byte_perm(w[j], tag, 0x3715);  // lanes (b1 << 8 | t1), (b3 << 8 | t3)
            acc = __vmaxu2(acc, __vmaxu2(e, o));
        }
    }
    return max(acc & 0xFFFFu, acc >> 16);
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
    __shared__ unsigned int wmx[S1_STAGES][S1_THREADS / 32];  // per warp of a tile: its blocks' maximum
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
        {
            static_assert(S1_TILE / 64 == S1_THREADS, "one block of the tile per thread");
            const uint32_t lb = (uint32_t)tid;
            const uint64_t P0 = T0 + 64ull * lb;
            const bool edge = P0 < a.lo || P0 + 64 > a.hi;
            const uint32_t key = block_key<false>(tb + 64 * lb, (lb >> 1) & 3u, inv, edge, P0, a.lo, a.hi);
            const uint32_t M = key >> 8;
            const uint64_t b = T0 / 64 + lb;
            if (b < a.nblk) {
                a.smax[b] = (uint8_t)M;
                a.sarg[b] = (uint8_t)(255u - (key & 0xFFu));
            }
            // 64 blocks (two warps) per 4 KiB superblock
            const uint32_t wm = __reduce_max_sync(FULL, M);
            if ((tid & 31) == 0 && wm) atomicMax(&supmax[s][lb >> 6], wm);
            if (a.spre) {
                // running maxima inside the superblock: warp scans here, the
                // other warp's maximum joined after the barrier below
                const int lane = tid & 31;
                uint32_t pf = M, sf = M;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t u = __shfl_up_sync(FULL, pf, d), v = __shfl_down_sync(FULL, sf, d);
                    if (lane >= d) pf = pf > u ? pf : u;
                    if (lane + d < 32) sf = sf > v ? sf : v;
                }
                if (lane == 0) wmx[s][tid >> 5] = wm;
                __syncthreads();
                const int wv = tid >> 5;
                if (wv & 1) {
                    const uint32_t o = wmx[s][wv - 1];
                    pf = pf > o ? pf : o;
                } else {
                    const uint32_t o = wmx[s][wv + 1];
                    sf = sf > o ? sf : o;
                }
                if (b < a.nblk) {
                    a.spre[b] = (uint8_t)pf;
                    a.ssuf[b] = (uint8_t)sf;
                }
            }
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

// Bytes of x in 16-bit lanes plus Kv = (0x8000 - v) * 0x00010001: bit 15 or
// 31 of either half of the result is set exactly when a byte is >= v
// (1 <= v <= 255), as b + 0x8000 - v carries into the lane's top bit.
__device__ __forceinline__ uint32_t ge_lanes(uint32_t x, uint32_t Kv) {
    return (__byte_perm(x, 0, 0x4240) + Kv) | (__byte_perm(x, 0, 0x4341) + Kv);
}

// Tiles of TB blocks (TB * 64 bytes of targets). TH = TB + 32 threads: one per
// stage block (the tile's blocks and up to 32 halo blocks) in the block-key
// pass, so that the halo costs no second round.
//
// Three barriers per tile: (1) the keys of every stage block are in shared
// memory, (2) the prefilter has listed its survivors, (3) the survivors'
// results are in the tile's target mask. The stage is refilled after (3), and
// every thread then writes its block's result with no further barrier: keys
// and masks are double-buffered by tile parity, so the next tile's key pass
// can start while slower warps still write this tile's results.
//
// Dynamic shared memory: 2 stages of (TB + 2*hb) * 64 bytes, then per tile
// parity the stage blocks' maxima and first positions, then 2 mbarriers.
template <int TB, int TH, int MINB>
__global__ void __launch_bounds__(TH, MINB) k_summary_maxp(SumLaunch a) {
    static_assert(TH >= TB + 32 && TB % 64 == 0 && TH % 32 == 0, "one thread per tile block, one halo warp");
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x;
    const uint32_t hb = a.halo_blocks;
    const uint32_t nb = TB + 2 * hb;  // blocks per stage
    const uint32_t sbytes = nb * 64;
    uint8_t* buf = smem;
    uint8_t* bmx = smem + 2 * sbytes;  // [parity][stage block] block maximum
    uint8_t* bfx = bmx + 2 * nb;       // [parity][stage block] first position of the maximum
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + ((2 * sbytes + 4 * nb + 15) & ~15u));
    __shared__ uint16_t slist[TB];        // tile blocks that passed the prefilter
    __shared__ uint32_t okm[2][TB / 32];  // [parity] tile blocks holding a target
    __shared__ unsigned int sn;
    if (blockIdx.x == 0 && tid == 0) reset_ctrl(a.ctrl);
    const uint64_t ntiles = (a.nblk + TB - 1) / TB;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint64_t g = gridDim.x;
    // stage block 0 stands for global block t * TB - hb (negative positions and
    // positions outside [glo, ghi) are not copied)
    auto issue = [&](uint64_t t, int s) {
        int64_t r0 = ((int64_t)(t * TB) - (int64_t)hb) * 64, r1 = r0 + (int64_t)sbytes;
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
    const uint32_t K = (w - 63) / 64;  // w >= 63
    const uint32_t li = (uint32_t)tid & 7u;
    uint32_t i = 0;
    for (uint64_t t = blockIdx.x; t < ntiles; t += g, i++) {
        const int s = i & 1;  // stage, and parity of the key and mask buffers
        const uint32_t par = (i >> 1) & 1u;
        if (!mbar_wait_bounded(&bar[s], par, a.timeout_ns)) {
            atomicOr(&a.ctrl->err, ERR_TIMEOUT);
            mbar_wait_bounded(&bar[0], par, a.timeout_ns);
            mbar_wait_bounded(&bar[1], par, a.timeout_ns);
            return;
        }
        const uint8_t* tb = buf + s * sbytes;
        uint8_t* bm = bmx + s * nb;
        uint8_t* bf = bfx + s * nb;
        uint32_t* okw = okm[s];
        const int64_t sb0 = (int64_t)(t * TB) - (int64_t)hb;  // global block of stage block 0
        // 1) block max and first position of the max, for every stage block.
        // (The buffers of this parity were last read by tile i-2, which every
        // thread finished before barrier (1) of tile i-1.)
        for (uint32_t sb = tid; sb < nb; sb += TH) {
            const int64_t gblk = sb0 + (int64_t)sb;
            uint32_t kf = 255u;  // blocks before position 0: max 0, first position 0
            if (gblk >= 0) {
                const uint64_t P0 = (uint64_t)gblk * 64;
                const bool edge = P0 < a.lo || P0 + 64 > a.hi;
                kf = block_key<false>(tb + 64 * sb, (sb >> 1) & 3u, 0u, edge, P0, a.lo, a.hi);
            }
            bm[sb] = (uint8_t)(kf >> 8);
            bf[sb] = (uint8_t)(255u - (kf & 0xFFu));
        }
        if (tid == 0) sn = 0;
        if (tid < TB / 32) okw[tid] = 0;
        __syncthreads();  // (1)
        // 2) prefilter, one thread per tile block: every block strictly inside
        // the maximum's window must stay below the maximum. Survivors (a small
        // share) are listed.
        if (tid < TB) {
            const uint32_t lb = (uint32_t)tid;
            const uint32_t sbi = hb + lb;
            const uint32_t v = bm[sbi];
            const uint32_t P = 64 * sbi + bf[sbi];  // the maximum's offset in the stage (> w)
            // interior blocks on each side (-1: the window ends inside the block)
            const int rl = (int)sbi - (int)((P - w) >> 6) - 1, rr = (int)((P + w) >> 6) - (int)sbi - 1;
            // both windows inside the data (checked here, while most blocks are
            // still candidates, to keep the survivors few)
            const uint64_t p = (t * TB + lb) * 64 + bf[sbi];
            bool pass = t * TB + lb < a.nblk && v != 0 && p >= a.lo + w && p + w < a.hi;
            // the K nearest blocks on each side lie inside the window wherever
            // the maximum sits: independent loads, no early exit
            uint32_t nm = 0;
            for (int d = 1; d <= (int)K; d++) nm = max(nm, max((uint32_t)bm[sbi - d], (uint32_t)bm[sbi + d]));
            pass = pass && nm < v;
            // then the (at most one) remaining interior block on each side
            const int d1 = (int)K + 1;
            if (d1 <= rl) nm = max(nm, (uint32_t)bm[sbi - d1]);
            if (d1 <= rr) nm = max(nm, (uint32_t)bm[sbi + d1]);
            pass = pass && nm < v;
            if (pass) slist[atomicAdd(&sn, 1u)] = (uint16_t)lb;
        }
        __syncthreads();  // (2)
        // 3) survivors, eight lanes each (lane li holds bytes 8li..8li+7 of a
        // block): no byte of the own block but the maximum, nor any byte of the
        // two partial end blocks that lies in the window, may reach the maximum.
        // Every warp runs the same number of rounds (the ballot takes whole warps).
        const uint32_t nsv = sn;
        for (uint32_t k0 = 0; k0 < nsv; k0 += TH / 8) {
            const uint32_t k = k0 + ((uint32_t)tid >> 3);
            const bool act = k < nsv;
            uint32_t lb = 0, hit = 0;
            if (act) {
                lb = slist[k];
                const uint32_t sbi = hb + lb;
                const uint32_t v = bm[sbi], f = bf[sbi];
                const uint64_t p = (t * TB + lb) * 64 + f;  // both windows inside the data (prefilter)
                const uint32_t o0 = (uint32_t)((p - w) & 63), o1 = (uint32_t)((p + w) & 63);
                const uint32_t s0 = (uint32_t)((int64_t)((p - w) >> 6) - sb0);
                const uint32_t s1 = (uint32_t)((int64_t)((p + w) >> 6) - sb0);
                const uint32_t Kv = (0x8000u - v) * 0x00010001u;
                const int b8 = 64 * (int)li;  // bit offset of the lane's first byte
                {
                    const uint2 q = *reinterpret_cast<const uint2*>(tb + 64 * sbi + 8 * li);
                    const uint32_t d = f - 8 * li;  // the maximum's byte among the lane's eight, if < 8
                    const uint32_t x0 = d < 4 ? q.x & ~(0xFFu << (8 * d)) : q.x;
                    const uint32_t x1 = (d - 4) < 4 ? q.y & ~(0xFFu << (8 * (d - 4))) : q.y;
                    hit |= ge_lanes(x0, Kv) | ge_lanes(x1, Kv);
                }
                if (s0 != sbi && bm[s0] >= v) {  // left end block: offsets >= o0
                    const uint2 q = *reinterpret_cast<const uint2*>(tb + 64 * s0 + 8 * li);
                    const int d = 8 * (int)o0 - b8;
                    const uint32_t x0 = q.x & __funnelshift_lc(0u, 0xFFFFFFFFu, (uint32_t)min(max(d, 0), 32));
                    const uint32_t x1 = q.y & __funnelshift_lc(0u, 0xFFFFFFFFu, (uint32_t)min(max(d - 32, 0), 32));
                    hit |= ge_lanes(x0, Kv) | ge_lanes(x1, Kv);
                }
                if (s1 != sbi && bm[s1] >= v) {  // right end block: offsets <= o1
                    const uint2 q = *reinterpret_cast<const uint2*>(tb + 64 * s1 + 8 * li);
                    const int d = b8 + 24 - 8 * (int)o1;
                    const uint32_t x0 = q.x & __funnelshift_rc(0xFFFFFFFFu, 0u, (uint32_t)min(max(d, 0), 32));
                    const uint32_t x1 = q.y & __funnelshift_rc(0xFFFFFFFFu, 0u, (uint32_t)min(max(d + 32, 0), 32));
                    hit |= ge_lanes(x0, Kv) | ge_lanes(x1, Kv);
                }
            }
            const uint32_t bal = __ballot_sync(FULL, (hit & 0x80008000u) != 0);
            if (act && li == 0 && ((bal >> (tid & 24)) & 0xFFu) == 0) atomicOr(&okw[lb >> 5], 1u << (lb & 31));
        }
        __syncthreads();  // (3)
        // the stage's bytes are no longer read: refill it with the tile after
        // next (from the halo warp, which has no result to write)
        if (tid == TH - 32) {
            uint64_t tn = t + 2 * g;
            if (tn < ntiles) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(tn, s);
            }
        }
        // 4) results: the target's offset or 0xFF per block, and the targets
        // per 4 KiB superblock (64 blocks: two mask words)
        if (tid < TB) {
            const uint32_t lb = (uint32_t)tid;
            const uint64_t gb = t * TB + lb;
            if (gb < a.nblk) a.smax[gb] = ((okw[lb >> 5] >> (lb & 31)) & 1u) ? bf[hb + lb] : (uint8_t)0xFFu;
        }
        if (tid < TB / 64) {
            const uint64_t q = t * (TB / 64) + tid;
            if (q < a.nsup) a.ssup[q] = (uint8_t)(__popc(okw[2 * tid]) + __popc(okw[2 * tid + 1]));
        }
    }
}

// ---- launchers -----------------------------------------------------------------

int summary_max_smem() { return S1_STAGES * S1_TILE + S1_STAGES * 8; }

// MAXP tiles: 512 blocks (32 KiB), 544 threads, 3 CTAs per SM (32 registers)
constexpr int MP_TILE_BLOCKS = 512, MP_THREADS = 544, MP_MIN_CTAS = 3;
static constexpr auto maxp_kernel = k_summary_maxp<MP_TILE_BLOCKS, MP_THREADS, MP_MIN_CTAS>;

int summary_maxp_smem(uint32_t halo_blocks) {
    uint32_t nb = MP_TILE_BLOCKS + 2 * halo_blocks;
    return (int)(((2 * nb * 64 + 4 * nb + 15) & ~15u) + 16);
}

uint32_t maxp_halo_blocks(uint32_t w) { return (w + 63) / 64 + 1; }

static int allow_summary_smem(int kind) {
    if (kind == SUM_MAXP) return launch_memo(300, 0, [](uint32_t) { return allow_max_smem(maxp_kernel); });
    if (kind == SUM_MAX_INV) return launch_memo(301, 0, [](uint32_t) { return allow_max_smem(k_summary_max<true>); });
    return launch_memo(302, 0, [](uint32_t) { return allow_max_smem(k_summary_max<false>); });
}

cudaError_t launch_summary(const SumLaunch& a, int kind, int grid, cudaStream_t st) {
    const int set = allow_summary_smem(kind);
    if (set != (int)cudaSuccess) return (cudaError_t)set;
    if (kind == SUM_MAXP) {
        maxp_kernel<<<grid, MP_THREADS, summary_maxp_smem(a.halo_blocks), st>>>(a);
    } else if (kind == SUM_MAX_INV) {
        k_summary_max<true><<<grid, S1_THREADS, summary_max_smem(), st>>>(a);
    } else {
        k_summary_max<false><<<grid, S1_THREADS, summary_max_smem(), st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_reset(Ctrl* ctrl, cudaStream_t st) {
    k_reset<<<1, 32, 0, st>>>(ctrl);
    return cudaGetLastError();
}

int summary_blocks_per_sm(int kind, uint32_t halo_blocks) {
    allow_summary_smem(kind);
    if (kind == SUM_MAXP)
        return launch_memo(310, halo_blocks, [](uint32_t hb) {
            int n = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, maxp_kernel, MP_THREADS, summary_maxp_smem(hb));
            return n > 0 ? n : 1;
        });
    return launch_memo(311, 0, [](uint32_t) {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_summary_max<false>, S1_THREADS, summary_max_smem());
        return n > 0 ? n : 1;
    });
}

uint64_t summary_tiles(int kind, uint64_t nblk) {
    return kind == SUM_MAXP ? (nblk + MP_TILE_BLOCKS - 1) / MP_TILE_BLOCKS : (nblk * 64 + S1_TILE - 1) / S1_TILE;
}

}  // namespace cdc
