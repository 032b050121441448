// prims.cu -- the two processing patterns of hashless chunking as standalone
// device operations over many byte ranges at once (include/cdc.h, cdc_ebs and
// cdc_rs):
//   Extreme Byte Search (Section 3.1): the maximum or minimum byte of a range
//     and the offset of its first occurrence;
//   Range Scan (Section 3.2): the first byte of a range that compares GT, LT,
//     GEQ, LEQ or EQ against a threshold.
// One warp per range: each lane takes a 16-byte granule per round (512 bytes
// per warp and round), bytes are compared in 16-bit lanes (a lane add that
// reaches bit 15 exactly when the byte is >= a threshold; native 16x2 max),
// the first hit comes from a ballot.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cdc.h"
#include "chain_logic.cuh"

namespace cdc {
namespace {

constexpr uint32_t FULLMASK = 0xFFFFFFFFu;

// bytes of granule g (16 bytes at base + 16 g) that lie in [a, b), others
// replaced by `fill` (a byte value that cannot win)
__device__ __forceinline__ void load_granule(const uint8_t* base, uint64_t g, uint64_t a, uint64_t b, uint32_t fill,
                                             uint32_t w[4]) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(base) + g);
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    const uint64_t p0 = g * 16;
    if (p0 >= a && p0 + 16 <= b) return;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint64_t wi = (p0 >> 2) + (uint64_t)k;
        const uint32_t keep = clip_word(0xFFFFFFFFu, wi, a, b);
        w[k] = (w[k] & keep) | (fill & ~keep);
    }
}

// bit 7 of each byte set where the byte satisfies the comparison with t
__device__ __forceinline__ uint32_t cmp_flags(uint32_t x, int cmp, uint32_t t) {
    switch (cmp) {
    case CDC_RS_GEQ: return ge_flags(x, ge_key(t));
    case CDC_RS_GT: return t >= 255 ? 0u : ge_flags(x, ge_key(t + 1));
    case CDC_RS_LEQ: return ge_flags(~x, ge_key(255 - t));  // b <= t  <=>  255 - b >= 255 - t
    case CDC_RS_LT: return t == 0 ? 0u : ge_flags(~x, ge_key(256 - t));
    default:  // EQ: b >= t and 255 - b >= 255 - t
        return ge_flags(x, ge_key(t)) & ge_flags(~x, ge_key(255 - t));
    }
}

__global__ void k_ebs(int op, const uint8_t* base, uint64_t lo, uint64_t len, const uint64_t* ranges, uint64_t n,
                      uint8_t* value, uint64_t* pos) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t inv = op == CDC_EBS_MIN ? 0xFFFFFFFFu : 0u;  // the minimum is the complement's maximum
    for (uint64_t q = warp; q < n; q += nwarps) {
        uint64_t a = ranges[2 * q], b = ranges[2 * q + 1];
        if (b > len) b = len;
        if (a >= b) {
            if (lane == 0) {
                value[q] = op == CDC_EBS_MIN ? 255 : 0;
                if (pos) pos[q] = ranges[2 * q];
            }
            continue;
        }
        a += lo;
        b += lo;
        const uint64_t g0 = a >> 4, g1 = (b - 1) >> 4;
        ByteMax m;
        for (uint64_t g = g0 + lane; g <= g1; g += 32) {
            uint32_t w[4];
            load_granule(base, g, a, b, inv, w);  // outside bytes read as 0 after the complement
#pragma unroll
            for (int k = 0; k < 4; k++) m.add(w[k] ^ inv);
        }
        const uint32_t M = __reduce_max_sync(FULLMASK, m.get());
        uint64_t first = a;  // every byte is the extreme when the maximum is 0
        if (pos && M > 0) {
            const uint32_t K = ge_key(M);
            for (uint64_t g0r = g0; g0r <= g1; g0r += 32) {
                const uint64_t g = g0r + lane;
                uint32_t hit = 0xFFFFFFFFu;
                if (g <= g1) {
                    uint32_t w[4];
                    load_granule(base, g, a, b, inv, w);
#pragma unroll
                    for (int k = 3; k >= 0; k--) {
                        const uint32_t f = ge_flags(w[k] ^ inv, K) & clip_word(0xFFFFFFFFu, g * 4 + k, a, b);
                        if (f) hit = 4u * (uint32_t)k + (uint32_t)((__ffs((int)f) - 1) >> 3);
                    }
                }
                const uint32_t bal = __ballot_sync(FULLMASK, hit != 0xFFFFFFFFu);
                if (bal) {
                    const int l = __ffs((int)bal) - 1;
                    const uint32_t hl = __shfl_sync(FULLMASK, hit, l);
                    first = (g0r + (uint64_t)l) * 16 + hl;
                    break;
                }
            }
        }
        if (lane == 0) {
            value[q] = (uint8_t)(op == CDC_EBS_MIN ? 255 - M : M);
            if (pos) pos[q] = first - lo;
        }
    }
}

__global__ void k_rs(int cmp, const uint8_t* base, uint64_t lo, uint64_t len, const uint64_t* ranges,
                     const uint8_t* thr, uint64_t n, uint64_t* pos) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t q = warp; q < n; q += nwarps) {
        uint64_t a = ranges[2 * q], b = ranges[2 * q + 1];
        if (b > len) b = len;
        const uint64_t end = ranges[2 * q + 1];
        uint64_t found = end;
        if (a < b) {
            const uint32_t t = thr[q];
            a += lo;
            b += lo;
            const uint64_t g0 = a >> 4, g1 = (b - 1) >> 4;
            for (uint64_t g0r = g0; g0r <= g1; g0r += 32) {
                const uint64_t g = g0r + lane;
                uint32_t hit = 0xFFFFFFFFu;
                if (g <= g1) {
                    uint32_t w[4];
                    load_granule(base, g, 0, ~0ull, 0, w);
#pragma unroll
                    for (int k = 3; k >= 0; k--) {
                        const uint32_t f = cmp_flags(w[k], cmp, t) & clip_word(0xFFFFFFFFu, g * 4 + k, a, b);
                        if (f) hit = 4u * (uint32_t)k + (uint32_t)((__ffs((int)f) - 1) >> 3);
                    }
                }
                const uint32_t bal = __ballot_sync(FULLMASK, hit != 0xFFFFFFFFu);
                if (bal) {
                    const int l = __ffs((int)bal) - 1;
                    const uint32_t hl = __shfl_sync(FULLMASK, hit, l);
                    found = (g0r + (uint64_t)l) * 16 + hl - lo;
                    break;
                }
            }
        }
        if (lane == 0) pos[q] = found;
    }
}

int grid_for(uint64_t n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t warps = (uint64_t)(sms > 0 ? sms : 148) * 64;  // 64 warps of 32 per SM at most
    const uint64_t w = n < warps ? n : warps;
    return (int)((w + 7) / 8);  // 8 warps per block
}

}  // namespace
}  // namespace cdc

using namespace cdc;

extern "C" cdc_status cdc_ebs(cdc_ebs_op op, const uint8_t* data, size_t len, const uint64_t* d_ranges, size_t n,
                              uint8_t* d_value, uint64_t* d_pos, cdc_stream stream) {
    if ((op != CDC_EBS_MAX && op != CDC_EBS_MIN) || (n && (!d_ranges || !d_value)) || (len && !data))
        return CDC_ERR_INVALID;
    if (n == 0) return CDC_OK;
    const uintptr_t p = (uintptr_t)data;
    const uint8_t* base = (const uint8_t*)(p & ~(uintptr_t)15);
    k_ebs<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((int)op, base, p & 15, len, d_ranges, n, d_value, d_pos);
    return cudaGetLastError() == cudaSuccess ? CDC_OK : CDC_ERR_CUDA;
}

extern "C" cdc_status cdc_rs(cdc_rs_cmp cmp, const uint8_t* data, size_t len, const uint64_t* d_ranges,
                             const uint8_t* d_thresholds, size_t n, uint64_t* d_pos, cdc_stream stream) {
    if ((int)cmp < 0 || (int)cmp > 4 || (n && (!d_ranges || !d_thresholds || !d_pos)) || (len && !data))
        return CDC_ERR_INVALID;
    if (n == 0) return CDC_OK;
    const uintptr_t p = (uintptr_t)data;
    const uint8_t* base = (const uint8_t*)(p & ~(uintptr_t)15);
    k_rs<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((int)cmp, base, p & 15, len, d_ranges, d_thresholds, n,
                                                        d_pos);
    return cudaGetLastError() == cudaSuccess ? CDC_OK : CDC_ERR_CUDA;
}

// ---- chunk fingerprints ------------------------------------------------------------
//
// A 128-bit non-cryptographic fingerprint per chunk, for deduplication
// reports: two 64-bit multiply-xorshift streams over the chunk's 4-byte words
// (taken at the chunk's own offsets, the last one zero-padded), each word
// mixed with its index; lanes of a warp take interleaved words and their
// states are folded in lane order, then with the length. Equal chunks give
// equal fingerprints; different chunks collide with negligible probability.

namespace cdc {
namespace {

__device__ __forceinline__ uint64_t fp_mix(uint64_t x) {
    x ^= x >> 31;
    x *= 0x7FB5D329728EA185ull;
    x ^= x >> 27;
    x *= 0x81DADEF4BC2DD44Dull;
    x ^= x >> 33;
    return x;
}

// chunk word j: bytes [s + 4j, s + 4j + 4) of the buffer at `base` (4-byte
// aligned), bytes at or past e read as 0; reads only words holding chunk bytes
__device__ __forceinline__ uint32_t chunk_word(const uint8_t* base, uint64_t s, uint64_t e, uint64_t j) {
    const uint64_t p = s + 4 * j;
    const uint64_t wi = p >> 2;
    const uint32_t sh = (uint32_t)(p & 3) * 8;
    const uint32_t* W = reinterpret_cast<const uint32_t*>(base);
    uint32_t lo = __ldg(W + wi), hi = 0;
    if (sh && ((wi + 1) << 2) < e) hi = __ldg(W + wi + 1);
    uint32_t v = sh ? __funnelshift_r(lo, hi, sh) : lo;
    if (p + 4 > e) v &= 0xFFFFFFFFu >> (8 * (uint32_t)(p + 4 - e));
    return v;
}

__global__ void k_fingerprint(const uint8_t* base, uint64_t lo, const uint64_t* bounds, uint64_t n, uint64_t* fp) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t c = warp; c < n; c += nwarps) {
        const uint64_t s = (c ? bounds[c - 1] : 0) + lo, e = bounds[c] + lo;
        const uint64_t nw = e > s ? (e - s + 3) / 4 : 0;
        uint64_t h1 = 0x243F6A8885A308D3ull ^ (uint64_t)lane, h2 = 0x13198A2E03707344ull ^ ((uint64_t)lane << 32);
        for (uint64_t j = lane; j < nw; j += 32) {
            const uint64_t x = ((uint64_t)chunk_word(base, s, e, j) << 32) | (uint32_t)j;
            h1 = fp_mix(h1 ^ x) + 0x9E3779B97F4A7C15ull;
            h2 = fp_mix(h2 + (x * 0xD6E8FEB86659FD93ull)) ^ (h2 >> 17);
        }
        // fold the 32 lane states in lane order (a fixed tree)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t a1 = __shfl_down_sync(0xFFFFFFFFu, h1, o), a2 = __shfl_down_sync(0xFFFFFFFFu, h2, o);
            if ((lane & (2 * o - 1)) == 0) {
                h1 = fp_mix(h1 * 0xFF51AFD7ED558CCDull + a1);
                h2 = fp_mix(h2 ^ (a2 * 0xC4CEB9FE1A85EC53ull));
            }
        }
        if (lane == 0) {
            const uint64_t L = e - s;
            fp[2 * c] = fp_mix(h1 ^ L);
            fp[2 * c + 1] = fp_mix(h2 + L * 0x9E3779B97F4A7C15ull);
        }
    }
}

// Byte shares of the two processing patterns (Section 3.3's composition),
// from the boundaries: one warp per chunk [s, e).
//   RAM: search w bytes (the rest for a tail of at most w), scan
//        e - max(s + w, s + min - 1).
//   AE:  the targets are the bytes beyond every earlier byte of the chunk
//        (positions p in [s, e) with B[p] beyond max B[s, p)); each target's
//        window search reads min(w, e - 1 - p) bytes, the scans from target to
//        target read (last target) - s.
// Targets come 32 bytes at a time: a warp max-scan of (byte + 1) gives the
// maximum before each lane, carried across rounds. Totals go to out[0..1]
// with one atomic per warp.
// the maximum byte of data[a, b) (b > a) and the last position holding it, for
// every lane of the warp
__device__ __forceinline__ uint32_t warp_max_last(const uint8_t* data, uint64_t a, uint64_t b, uint64_t& at) {
    const int lane = threadIdx.x & 31;
    uint32_t best = 0;
    uint64_t pos = a;
    for (uint64_t i = a + (uint64_t)lane; i < b; i += 32) {
        const uint32_t v = data[i];
        if (v >= best) {
            best = v;
            pos = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint32_t ob = __shfl_xor_sync(FULLMASK, best, o);
        const uint64_t op = __shfl_xor_sync(FULLMASK, pos, o);
        if (ob > best || (ob == best && op > pos)) {
            best = ob;
            pos = op;
        }
    }
    at = pos;
    return best;
}

// the first position in [a, b) whose byte is greater than t, or b
__device__ __forceinline__ uint64_t warp_first_gt(const uint8_t* data, uint64_t a, uint64_t b, uint32_t t) {
    const int lane = threadIdx.x & 31;
    for (uint64_t b0 = a; b0 < b; b0 += 32) {
        const uint64_t i = b0 + (uint64_t)lane;
        const unsigned hit = __ballot_sync(FULLMASK, i < b && data[i] > t);
        if (hit) return b0 + (uint64_t)(__ffs(hit) - 1);
    }
    return b;
}

// MAXP shares of the chunk from s, the procedure of Section 3.3 run by the
// whole warp: GT scans for a byte above the maximum of its left window (that
// maximum's last position m bounds the scan at m + w, where m leaves the
// window), then a search of the right window of each byte the scan stops at
__device__ void maxp_chunk_shares(const uint8_t* data, uint64_t len, uint64_t s, uint32_t w, uint32_t mn,
                                  uint32_t mx, unsigned long long& ebs, unsigned long long& rs) {
    const uint64_t L = len - s < mx ? len : s + mx;
    const uint64_t cend = len > w ? (L < len - w ? L : len - w) : 0;
    uint64_t p = s + mn - 1 > w ? s + mn - 1 : w;
    while (p < cend) {
        uint64_t m;
        const uint32_t lmax = warp_max_last(data, p - w, p, m);
        ebs += w;
        const uint64_t stop = m + w + 1 < cend ? m + w + 1 : cend;
        const uint64_t q = warp_first_gt(data, p, stop, lmax);
        if (q >= stop) {
            rs += stop - p;
            p = stop;
            continue;
        }
        rs += q - p + 1;
        uint64_t at;
        const uint32_t rmax = warp_max_last(data, q + 1, q + w + 1, at);
        ebs += w;
        if (data[q] > rmax) break;
        p = q + 1;
    }
}

__global__ void k_byte_shares(int alg, const uint8_t* data, uint64_t len, const uint64_t* bounds, uint64_t n,
                              uint32_t w, uint32_t mn, uint32_t mx, unsigned long long* out) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t inv = alg == CDC_AE_MIN ? 0xFFu : 0u;
    unsigned long long ebs = 0, rs = 0;
    for (uint64_t c = warp; c < n; c += nwarps) {
        const uint64_t s = c ? bounds[c - 1] : 0, e = bounds[c];
        if (e <= s || e > len) continue;
        if (alg == CDC_MAXP) {
            unsigned long long ce = 0, cr = 0;
            maxp_chunk_shares(data, len, s, w, mn, mx, ce, cr);
            if (lane == 0) {
                ebs += ce;
                rs += cr;
            }
            continue;
        }
        if (alg == CDC_RAM) {
            if (lane == 0) {
                if (len - s <= w) {
                    ebs += len - s;
                } else {
                    ebs += w;
                    const uint64_t from = s + w > s + mn - 1 ? s + w : s + mn - 1;
                    if (e > from) rs += e - from;
                }
            }
            continue;
        }
        uint32_t carry = 0;   // (max byte so far) + 1; 0 before the first byte
        uint64_t last = s;    // last target seen by this lane
        for (uint64_t b0 = s; b0 < e; b0 += 32) {
            const uint64_t p = b0 + (uint64_t)lane;
            const uint32_t v = p < e ? ((uint32_t)(data[p] ^ inv) + 1u) : 0u;
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(FULLMASK, incl, o);
                if (lane >= o) incl = max(incl, t);
            }
            uint32_t before = __shfl_up_sync(FULLMASK, incl, 1);
            if (lane == 0) before = 0;
            before = max(before, carry);
            if (v > before) {  // a target
                const uint64_t room = e - 1 - p;
                ebs += room < w ? room : w;
                last = p;
            }
            carry = max(carry, __shfl_sync(FULLMASK, incl, 31));
        }
        // the chunk's last target: the largest position any lane saw
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t t = __shfl_xor_sync(FULLMASK, last, o);
            last = t > last ? t : last;
        }
        if (lane == 0) rs += last - s;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ebs += __shfl_xor_sync(FULLMASK, ebs, o);
        rs += __shfl_xor_sync(FULLMASK, rs, o);
    }
    if (lane == 0 && (ebs || rs)) {
        atomicAdd(&out[0], ebs);
        atomicAdd(&out[1], rs);
    }
}

// chunk sizes b[i] - b[i-1] (b[-1] = 0) counted in n_bins bins of bin_width
// bytes, the last bin taking every larger size; per-block counts in shared
// memory, then one atomic per bin and block
__global__ void k_size_hist(const uint64_t* bounds, uint64_t n, uint64_t bin_width, uint32_t n_bins,
                            unsigned long long* hist) {
    extern __shared__ unsigned int sh[];
    for (uint32_t i = threadIdx.x; i < n_bins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < n; c += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s = c ? bounds[c - 1] : 0, e = bounds[c];
        const uint64_t size = e > s ? e - s : 0;
        const uint64_t b = size / bin_width;
        atomicAdd(&sh[b < n_bins ? (uint32_t)b : n_bins - 1], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n_bins; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

}  // namespace
}  // namespace cdc

extern "C" cdc_status cdc_size_histogram(const uint64_t* d_bounds, size_t n, uint64_t bin_width, uint32_t n_bins,
                                         uint64_t* d_hist, cdc_stream stream) {
    if (!d_hist || (n && !d_bounds) || bin_width == 0 || n_bins == 0 || n_bins > 8192) return CDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_hist, 0, n_bins * sizeof(uint64_t), st) != cudaSuccess) return CDC_ERR_CUDA;
    if (n == 0) return CDC_OK;
    uint64_t grid = (n + 255) / 256;
    if (grid > 1024) grid = 1024;
    cdc::k_size_hist<<<(unsigned)grid, 256, n_bins * sizeof(unsigned int), st>>>(
        d_bounds, n, bin_width, n_bins, reinterpret_cast<unsigned long long*>(d_hist));
    return cudaGetLastError() == cudaSuccess ? CDC_OK : CDC_ERR_CUDA;
}

extern "C" cdc_status cdc_byte_shares(cdc_alg alg, cdc_params p, const uint8_t* data, size_t len,
                                      const uint64_t* d_bounds, size_t n, uint64_t* d_out, cdc_stream stream) {
    if ((int)alg < 0 || (int)alg > 3 || !d_out || (n && !d_bounds) || (len && !data)) return CDC_ERR_INVALID;
    if (p.w < 1 || p.min < 1 || p.min > p.max) return CDC_ERR_INVALID;
    if ((alg == CDC_AE || alg == CDC_AE_MIN) && p.min > p.w + 1) return CDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_out, 0, 2 * sizeof(uint64_t), st) != cudaSuccess) return CDC_ERR_CUDA;
    if (n == 0) return CDC_OK;
    cdc::k_byte_shares<<<cdc::grid_for(n), 256, 0, st>>>((int)alg, data, len, d_bounds, n, p.w, p.min, p.max,
                                                          reinterpret_cast<unsigned long long*>(d_out));
    return cudaGetLastError() == cudaSuccess ? CDC_OK : CDC_ERR_CUDA;
}

extern "C" cdc_status cdc_fingerprint(const uint8_t* data, size_t len, const uint64_t* d_bounds, size_t n,
                                      uint64_t* d_fp, cdc_stream stream) {
    if ((n && (!d_bounds || !d_fp)) || (len && !data)) return CDC_ERR_INVALID;
    if (n == 0) return CDC_OK;
    const uintptr_t p = (uintptr_t)data;
    const uint8_t* base = (const uint8_t*)(p & ~(uintptr_t)3);
    k_fingerprint<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(base, p & 3, d_bounds, n, d_fp);
    return cudaGetLastError() == cudaSuccess ? CDC_OK : CDC_ERR_CUDA;
}
