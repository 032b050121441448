// graph.cu -- stage 2 in candidate-graph form: the chunk chain of one stream,
// bit-exact, with work in proportion to the candidate cut positions rather
// than to the chains a speculation has to follow.
//
// The chunk chain s_{i+1} = next(s_i) (Section 3.3: each algorithm handles
// one chunk at a time) only ever ends a chunk at a candidate position (a
// natural cut, graph_logic.cuh), at a forced cut or inside a quiet stretch.
// So the chain is a path in the graph y -> F(y) over the candidates, F(y)
// being the next candidate on the chain that starts at y. Segments of S bytes
// (S >= max) hold slots of `cap` candidates each:
//
//  k_gcand   one CTA per segment: enumerates the segment's candidates from the
//            block summaries (raw bytes only for blocks that can hold one),
//            in increasing order, into the segment's slot.
//  k_glocal  one CTA per segment: F(y) for every candidate of the segment from
//            the sorted candidate lists of the segment and the next one
//            (list_next; stepping the chain only for forced cuts and quiet
//            runs), then pointer jumping in shared memory: for every
//            candidate, the first candidate on its chain past the segment
//            (an id in a later segment) and the chunk ends up to it.
//  k_gunit   (when the segments form several units of G): the same "first
//            candidate past the unit" for every candidate of a unit's first
//            segment, by following the segment exits.
//  k_gtop    one thread follows the true chain from the first byte over the
//            unit tables (or over the segments, when there is one unit),
//            recording each unit's entry and the boundaries before it.
//  k_gdesc   one thread per unit follows the chain through its segments,
//            recording each segment's entry and output offset.
//  k_gemit   one thread per segment replays its part of the true chain from the
//            stored F steps and writes the boundaries.
// No kernel waits on another CTA. Candidates beyond a full slot (inputs with
// more than cap candidates in S bytes) are handled by stepping the chain
// (GID_SLOW): slower, still exact.
#include "cdc_device.cuh"
#include "cdc_launch.h"
#include "graph_logic.cuh"
#include "warp_rules.cuh"

namespace cdc {

constexpr int GC_THREADS = 256;  // k_gcand
// k_glocal runs 512 threads per segment when a segment has up to 4096 slots,
// 256 (two CTAs per SM) when it has up to 2048; each thread takes up to
// GL_PER candidates in the jumping rounds
constexpr int GL_PER = 8;
constexpr uint32_t GL_EXIT = 0xFFFFFFFFu;
constexpr uint32_t GL_PEND = 0xFFFFFFFEu;  // F not yet known (k_glocal)
constexpr int GE_BUF = 256;      // k_gemit: boundaries buffered before a store

__device__ __forceinline__ uint64_t g_seg_lo(const GraphLaunch& A, uint32_t k) { return A.lo + (uint64_t)k * A.S; }
__device__ __forceinline__ uint64_t g_seg_hi(const GraphLaunch& A, uint32_t k) {
    const uint64_t e = A.lo + (uint64_t)(k + 1) * A.S;
    return e < A.hi ? e : A.hi;
}
__device__ __forceinline__ uint32_t g_seg_of(const GraphLaunch& A, uint64_t y) { return (uint32_t)((y - A.lo) / A.S); }
__device__ __forceinline__ uint32_t g_slot_n(const GraphLaunch& A, uint32_t k) {
    const uint32_t n = A.cnum[k];
    return n < A.cap ? n : A.cap;
}
// position of candidate id (id < GID_NONE)
__device__ __forceinline__ uint64_t g_pos(const GraphLaunch& A, uint32_t id) {
    return g_seg_lo(A, id / A.cap) + A.cpos[id];
}

// a consistency check failed: flag it (the host reports CDC_ERR_INTERNAL)
__device__ __forceinline__ void g_fail(const GraphLaunch& A, uint64_t info) {
    atomicOr(&A.ctrl->err, ERR_INTERNAL);
    A.ctrl->err_info = info;
}

// first index in p[0, n) whose value is >= v
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* p, uint32_t n, uint32_t v) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (p[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// id of the candidate at position y (a candidate of segment k), or GID_SLOW
// when it lies beyond the segment's slot
__device__ uint32_t g_find(const GraphLaunch& A, uint32_t k, uint64_t y) {
    const uint32_t n = g_slot_n(A, k);
    const uint32_t* p = A.cpos + (uint64_t)k * A.cap;
    const uint32_t r = (uint32_t)(y - g_seg_lo(A, k));
    const uint32_t i = lower_bound_u32(p, n, r);
    return (i < n && p[i] == r) ? k * A.cap + i : GID_SLOW;
}

// Follow the chain from candidate `id` by F steps until the first candidate
// with a slot in a later segment (or the end); used where a slot overflowed.
template <int RULE>
__device__ unsigned long long g_slow_hop(const GraphLaunch& A, uint32_t id) {
    const Prm P{A.w, A.mn, A.mx};
    const RawView R{A.base, A.inv};
    const SumView S{A.smax, A.sarg, nullptr, nullptr, 0, 0, A.ssup};
    const PreSuf T{A.spre, A.ssuf};
    const uint32_t k = id / A.cap;
    uint64_t y = g_pos(A, id);
    unsigned long long acc = 0;
    for (;;) {
        uint32_t c;
        const uint64_t e = cand_next_t<RULE>(S, T, R, P, A.flo, A.hi, y, &c);
        acc += c;
        if (e >= A.hi) return (acc << 32) | GID_END;
        const uint32_t k2 = g_seg_of(A, e);
        if (k2 > k) {
            const uint32_t f = g_find(A, k2, e);
            if (f != GID_SLOW) return (acc << 32) | f;
        }
        y = e;
    }
}

// (ends << 32) | id of the first candidate past candidate id's segment
template <int RULE>
__device__ __forceinline__ unsigned long long g_hop(const GraphLaunch& A, uint32_t id) {
    const unsigned long long v = A.cex[id];
    if ((uint32_t)v == GID_SLOW) return g_slow_hop<RULE>(A, id);
    return v;
}

// ---- k_gcand: candidates of each segment, in order ------------------------------
//
// A candidate's byte is at least the maximum of the whole blocks its window
// covers, and every source byte of a block shares those blocks but for two
// partial ones; so per block the maximum L of the whole blocks common to all
// its bytes' windows (two or three reads of the running maxima inside
// superblocks) rejects most blocks without reading them. The
// blocks that pass are listed, then read one per thread: bytes >= max(L, 1) are
// flagged with packed compares; a flagged byte is a candidate if no flagged byte
// before it (RAM) or after it (AE) in the block is greater and the partial
// block at the far end of its window holds no greater byte (block maxima
// first, raw bytes only where a block maximum is greater).

constexpr uint32_t GC_CH = 2048;                 // source blocks per chunk
constexpr uint32_t GC_KMAX = 1024;               // longest whole-block window whose far end is staged
constexpr uint32_t GC_ST = GC_CH + GC_KMAX + 256;  // staged blocks per chunk: the chunk, a halo on one side, 64-block alignment

struct GcShared {
    __align__(16) uint8_t a[GC_ST];  // block maxima of [st0, st1)
    __align__(16) uint8_t pre[GC_ST];  // their running maxima inside superblocks
    __align__(16) uint8_t suf[GC_ST];
    __align__(16) uint8_t sup[GC_ST / 64 + 32];  // superblock maxima of [st0 / 64, ...)
    uint8_t cv[GC_CH];     // listed block: the byte of its candidates if they share one, else 0
    uint16_t list[GC_CH];  // passing blocks (offsets from the chunk start)
    uint8_t lval[GC_CH];   // their L
    unsigned long long mask[GC_CH];
    uint32_t wsum[GC_THREADS / 32];
    uint32_t nlist;
};

// exclusive prefix of v over the block's threads (in thread order); *tot = sum
__device__ __forceinline__ uint32_t gc_scan(uint32_t v, uint32_t* wsum, uint32_t* tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    uint32_t pre = 0, sum = 0;
#pragma unroll
    for (int k = 0; k < GC_THREADS / 32; k++) {
        const uint32_t x = wsum[k];
        if (k < wid) pre += x;
        sum += x;
    }
    __syncthreads();  // wsum is reused by the caller's next scan
    *tot = sum;
    return pre + incl - v;
}

// is any byte of [p, e) above x? (block maxima first: staged a[] for blocks in
// [st0, st1), else global; raw bytes only for partial blocks above x)
__device__ __forceinline__ bool gc_exceeds(const GraphLaunch& A, const RawView& R, const uint8_t* a, uint64_t st0,
                                           uint64_t st1, uint64_t p, uint64_t e, uint32_t x) {
    for (uint64_t blk = p >> 6; p < e && blk <= (e - 1) >> 6; blk++) {
        const uint32_t m = (blk >= st0 && blk < st1) ? a[blk - st0] : A.smax[blk];
        if (m <= x) continue;
        const uint64_t b0 = blk << 6;
        const uint64_t l = umax64(p, b0), h = umin64(e, b0 + 64);
        if (l == b0 && h == b0 + 64) return true;
        if (raw_max(R, l, h) > x) return true;
    }
    return false;
}

// maximum of the whole blocks [fb, lb) from the staged running maxima (the
// blocks lie in [st0, st1), st0 a multiple of 64)
__device__ __forceinline__ uint32_t gc_whole(const GcShared& sh, uint64_t st0, uint64_t fb, uint64_t lb) {
    const uint64_t q0 = fb >> 6, q1 = (lb - 1) >> 6;
    uint32_t M;
    if (q0 == q1) {
        if ((fb & 63) == 0) return sh.pre[lb - 1 - st0];
        if ((lb & 63) == 0) return sh.suf[fb - st0];
        M = 0;
        for (uint64_t x = fb; x < lb; x++) M = max(M, (uint32_t)sh.a[x - st0]);
        return M;
    }
    M = max((uint32_t)sh.suf[fb - st0], (uint32_t)sh.pre[lb - 1 - st0]);
    for (uint64_t q = q0 + 1; q < q1; q++) M = max(M, (uint32_t)sh.sup[q - (st0 >> 6)]);
    return M;
}

template <int RULE>
__global__ void __launch_bounds__(GC_THREADS) k_gcand(GraphLaunch A) {
    __shared__ GcShared sh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const Prm P{A.w, A.mn, A.mx};
    const RawView R{A.base, A.inv};
    const SumView S{A.smax, A.sarg, nullptr, nullptr, 0, 0, A.ssup};
    uint64_t qa0, qb0;
    cand_source_range<RULE>(P, A.flo, A.hi, &qa0, &qb0);
    const uint64_t shf = cand_shift<RULE>(P);
    {
        // candidates lie past the chain's start (the first slot holds the start)
        const uint64_t qmin = A.lo + 1 > shf ? A.lo + 1 - shf : 0;
        if (qa0 < qmin) qa0 = qmin;
        if (qb0 < qa0) qb0 = qa0;
    }
    const uint64_t w = A.w;
    // whole blocks of the window common to a block's bytes: RAM [b - K, b),
    // AE [b + 1, b + 1 + K); MAXP reads its targets directly
    uint32_t K = 0;
    if (RULE == RULE_RAM) K = w >= 126 ? (uint32_t)((w - 126 + 63) >> 6) : 0;
    if (RULE == RULE_AE) K = (uint32_t)((w + 1) >> 6) - 1;
    // blocks staged around a chunk: its blocks and, for windows of up to GC_KMAX
    // whole blocks, the partial blocks at the far end of its bytes' windows
    const bool table = K > 0 && K <= GC_KMAX;
    const uint32_t pre = (table && RULE == RULE_RAM) ? K + 2 : 0;
    const uint32_t post = (table && RULE == RULE_AE) ? K + 3 : 0;
    const PreSuf V{A.spre, A.ssuf};
    for (uint32_t seg = blockIdx.x; seg < A.nseg; seg += gridDim.x) {
        const uint64_t a = g_seg_lo(A, seg), b = g_seg_hi(A, seg);
        uint32_t* slot = A.cpos + (uint64_t)seg * A.cap;
        uint32_t run = 0;
        if (seg == 0) {
            if (tid == 0) slot[0] = 0;  // the chain starts at the first byte
            run = 1;
        }
        if (tid == 0) {
            A.sent[seg] = GID_NONE;
            if (seg % A.G == 0) A.uent[seg / A.G] = GID_NONE;
            if (seg == 0) {
                A.cval[0] = 0;
                A.cfar[0] = 0;
                A.ticket[0] = 0;
                A.ticket[1] = 0;
            }
        }
        uint64_t qa = a >= shf ? a - shf : 0, qb = b >= shf ? b - shf : 0;
        if (qa < qa0) qa = qa0;
        if (qb > qb0) qb = qb0;
        const uint64_t bl = qa < qb ? (qb - 1) >> 6 : 0;
        for (uint64_t cb0 = qa >> 6; qa < qb && cb0 <= bl; cb0 += GC_CH) {
            const uint64_t cb1 = umin64(cb0 + GC_CH, bl + 1);
            const uint32_t nb = (uint32_t)(cb1 - cb0);
            long long c0 = A.stats ? clock64() : 0;
            uint64_t st0 = 0, st1 = 0;
            if (RULE != RULE_MAXP) {
                st0 = (cb0 >= pre ? cb0 - pre : 0) & ~63ull;
                st1 = (cb1 + post + 63) & ~63ull;
                for (uint64_t q = tid; q < (st1 - st0) / 16; q += GC_THREADS) {
                    reinterpret_cast<uint4*>(sh.a)[q] = reinterpret_cast<const uint4*>(A.smax + st0)[q];
                    if (A.spre) {
                        reinterpret_cast<uint4*>(sh.pre)[q] = reinterpret_cast<const uint4*>(A.spre + st0)[q];
                        reinterpret_cast<uint4*>(sh.suf)[q] = reinterpret_cast<const uint4*>(A.ssuf + st0)[q];
                    }
                }
                for (uint64_t q = tid; q < (st1 - st0) / 64; q += GC_THREADS) sh.sup[q] = A.ssup[st0 / 64 + q];
                __syncthreads();
            }
            if (tid == 0) sh.nlist = 0;
            __syncthreads();
            long long c1 = A.stats ? clock64() : 0;
            // 1. list the blocks that can hold a candidate, in order
            for (uint32_t r0 = 0; r0 < nb; r0 += GC_THREADS) {
                const uint32_t o = r0 + (uint32_t)tid;
                const uint64_t blk = cb0 + o;
                bool pass = false;
                uint32_t L = 0;
                if (o < nb) {
                    if (RULE == RULE_MAXP) {
                        pass = A.smax[blk] != 0xFFu;
                    } else {
                        const uint32_t bm = sh.a[blk - st0];
                        if (K > 0) {
                            const uint64_t ws = RULE == RULE_RAM ? blk - K : blk + 1;  // window [ws, ws + K)
                            L = table && A.spre ? gc_whole(sh, st0, ws, ws + K) : whole_max(S, V, ws, ws + K);
                        }
                        pass = bm != 0 && bm >= L;
                    }
                }
                const uint32_t bal = __ballot_sync(FULL, pass);
                if (lane == 0) sh.wsum[wid] = __popc(bal);
                __syncthreads();
                uint32_t wp = sh.nlist, tot = 0;
#pragma unroll
                for (int k = 0; k < GC_THREADS / 32; k++) {
                    const uint32_t x = sh.wsum[k];
                    if (k < wid) wp += x;
                    tot += x;
                }
                if (pass) {
                    const uint32_t at = wp + __popc(bal & ((1u << lane) - 1));
                    sh.list[at] = (uint16_t)o;
                    sh.lval[at] = (uint8_t)L;
                }
                __syncthreads();
                if (tid == 0) sh.nlist += tot;
                __syncthreads();
            }
            const uint32_t nl = sh.nlist;
            long long c2 = A.stats ? clock64() : 0;
            // 2. the candidates of each listed block
            for (uint32_t e = tid; e < nl; e += GC_THREADS) {
                const uint64_t blk = cb0 + sh.list[e];
                const uint64_t b0 = blk << 6;
                const uint32_t oa = qa > b0 ? (uint32_t)(qa - b0) : 0u;
                const uint32_t ob = qb < b0 + 64 ? (uint32_t)(qb - b0) : 64u;
                unsigned long long m = 0;
                uint32_t cv = 0, cv_mixed = 0;  // the candidates' common byte
                if (RULE == RULE_MAXP) {
                    const uint32_t o = A.smax[blk];
                    if (o >= oa && o < ob) m = 1ull << o;
                } else {
                    uint32_t wd[16];
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const uint64_t g = (b0 >> 4) + (uint64_t)k;
                        if ((g << 4) >= (A.flo & ~15ull) && (g << 4) < A.hi) {
                            const uint4 v = __ldg(reinterpret_cast<const uint4*>(A.base) + g);
                            wd[4 * k] = v.x ^ A.inv; wd[4 * k + 1] = v.y ^ A.inv;
                            wd[4 * k + 2] = v.z ^ A.inv; wd[4 * k + 3] = v.w ^ A.inv;
                        } else {
                            wd[4 * k] = wd[4 * k + 1] = wd[4 * k + 2] = wd[4 * k + 3] = 0;
                        }
                    }
                    const uint32_t L = sh.lval[e];
                    const uint32_t Kg = ge_key(L > 1 ? L : 1u);
                    uint32_t run_max = 0;
                    if (RULE == RULE_RAM) {
                        const uint64_t h1 = (blk - K) << 6;  // the window's bytes before its whole blocks
#pragma unroll
                        for (int i = 0; i < 16; i++) {
                            uint32_t f = ge_flags(wd[i], Kg);
                            while (f) {
                                const uint32_t k = (uint32_t)(__ffs((int)f) - 1) >> 3;
                                f &= f - 1;
                                const uint32_t o = 4u * (uint32_t)i + k, x = (wd[i] >> (8 * k)) & 0xFFu;
                                if (o >= oa && o < ob && x >= run_max &&
                                    (x == 255u || !gc_exceeds(A, R, sh.a, st0, st1, b0 + o - w, h1, x))) {
                                    m |= 1ull << o;
                                    cv_mixed |= cv != 0 && cv != x;
                                    cv = x;
                                }
                                if (x > run_max) run_max = x;
                            }
                        }
                    } else {
                        const uint64_t t0 = (blk + 1 + K) << 6;  // the window's bytes past its whole blocks
#pragma unroll
                        for (int i = 15; i >= 0; i--) {
                            uint32_t f = ge_flags(wd[i], Kg);
                            while (f) {
                                const uint32_t bit = 31u - (uint32_t)__clz((int)f);
                                f &= ~(1u << bit);
                                const uint32_t k = bit >> 3;
                                const uint32_t o = 4u * (uint32_t)i + k, x = (wd[i] >> (8 * k)) & 0xFFu;
                                if (o >= oa && o < ob && x >= run_max &&
                                    (x == 255u || !gc_exceeds(A, R, sh.a, st0, st1, t0, b0 + o + w + 1, x))) {
                                    m |= 1ull << o;
                                    cv_mixed |= cv != 0 && cv != x;
                                    cv = x;
                                }
                                if (x > run_max) run_max = x;
                            }
                        }
                    }
                }
                sh.mask[e] = m;
                sh.cv[e] = cv_mixed ? 0 : (uint8_t)cv;
            }
            __syncthreads();
            long long c3 = A.stats ? clock64() : 0;
            // 3. positions, in block order
            const uint32_t per = (nl + GC_THREADS - 1) / GC_THREADS;
            const uint32_t e0 = (uint32_t)tid * per, e1 = e0 + per < nl ? e0 + per : nl;
            uint32_t cnt = 0;
            for (uint32_t e = e0; e < e1; e++) cnt += (uint32_t)__popcll(sh.mask[e]);
            uint32_t tot;
            uint32_t at = run + gc_scan(cnt, sh.wsum, &tot);
            for (uint32_t e = e0; e < e1; e++) {
                unsigned long long m = sh.mask[e];
                const uint64_t b0 = (cb0 + sh.list[e]) << 6;
                const uint32_t cve = sh.cv[e];
                while (m) {
                    const int o = __ffsll((long long)m) - 1;
                    m &= m - 1;
                    if (at < A.cap) {
                        slot[at] = (uint32_t)((b0 + (uint64_t)o + shf) - a);
                        A.cval[(uint64_t)seg * A.cap + at] =
                            RULE == RULE_MAXP ? 0 : (uint8_t)(cve ? cve : R.byte(b0 + (uint64_t)o));
                        A.cfar[(uint64_t)seg * A.cap + at] = 0;
                    }
                    at++;
                }
            }
            run += tot;
            __syncthreads();  // shared arrays are reused by the next chunk
            if (A.stats && tid == 0) {
                const long long c4 = clock64();
                atomicAdd(&A.stats[GST_CC_STAGE], (unsigned long long)(c1 - c0));
                atomicAdd(&A.stats[GST_CC_LIST], (unsigned long long)(c2 - c1));
                atomicAdd(&A.stats[GST_CC_BLOCKS], (unsigned long long)(c3 - c2));
                atomicAdd(&A.stats[GST_CC_WRITE], (unsigned long long)(c4 - c3));
                atomicAdd(&A.stats[GST_CC_LISTED], (unsigned long long)nl);
                atomicMax(&A.stats[GST_CC_MAX], (unsigned long long)(c4 - c0));
            }
        }
        if (tid == 0) A.cnum[seg] = run;
    }
}

// ---- k_glocal: F of every candidate, then the segment exits by jumping ----------
//
// One CTA per segment, segments taken in order from a ticket counter (a
// segment whose chains cross a long quiet stretch holds one CTA, not a
// static share of the grid). The segment's candidates and the next
// segment's are listed in shared memory with their bytes, next to the block
// maxima around them and their running maxima inside superblocks, so F of a candidate
// is a binary search, one or two window maxima and a comparison
// (list_next); only forced cuts, quiet runs and list overflows step the chain
// (cand_next_t). Then pointer jumping in shared memory gives every candidate
// the first candidate on its chain past the segment and the chunk ends up to it.

// shared memory of k_glocal: lists of 2 cap entries (positions, bytes), three
// jumping arrays of cap words, and the staged block maxima with their running
// maxima inside superblocks (`win` bytes each)
__host__ __device__ inline uint32_t gl_stage_off(uint32_t cap) { return (22u * cap + cap / 16u + 15u) & ~15u; }
// (the queue of candidates whose F steps the chain, one word per candidate, follows)
__host__ __device__ inline uint32_t gl_queue_off(int rule, uint32_t cap, uint32_t win) {
    return gl_stage_off(cap) + (rule == RULE_MAXP ? 0u : 3u * win);
}
int graph_local_smem(int rule, uint32_t cap, uint32_t win) {
    return (int)(gl_queue_off(rule, cap, win) + 4u * cap);
}

// Is position y a candidate (is_cand), decided by the whole warp
template <int RULE>
__device__ bool w_is_cand(const SumView& S, const RawView& R, const Prm& P, uint64_t lo, uint64_t hi, uint64_t y) {
    uint64_t a, b;
    cand_source_range<RULE>(P, lo, hi, &a, &b);
    const uint64_t sh = cand_shift<RULE>(P);
    if (y < sh) return false;
    const uint64_t q = y - sh;
    if (q < a || q >= b) return false;
    if (RULE == RULE_MAXP) return S.m(q >> 6) == (uint32_t)(q & 63);
    const uint32_t x = R.byte(q);
    if (x == 0) return false;
    if (x == 255) return true;
    if (RULE == RULE_RAM) return w_range_max(S, R, q - P.w, q) <= x;
    return w_range_max(S, R, q + 1, q + P.w + 1) <= x;
}

// Range Scan (GEQ) over [from, to) for the whole warp: whole 4 KiB superblocks
// whose maximum is below M are skipped 32 at a time (a ballot over their
// summaries), the rest as w_first_geq. Equals first_geq.
__device__ uint64_t w_first_geq_far(const SumView& S, const RawView& R, uint64_t from, uint64_t to, uint32_t M,
                                    uint32_t* val) {
    uint64_t p = from;
    while (p < to) {
        if ((p & 4095) == 0 && S.sup && p + 4096 <= to) {
            const uint64_t q0 = p >> 12, qn = (to >> 12) - q0;  // whole superblocks before `to`
            const bool hit = (uint64_t)lane_id() < qn && S.sup[q0 + lane_id()] >= M;
            const uint32_t bal = __ballot_sync(FULL, hit);
            if (bal == 0) {
                p = (q0 + umin64(qn, 32)) << 12;
                continue;
            }
            const int l = __ffs((int)bal) - 1;
            if (l > 0) {
                p = (q0 + (uint64_t)l) << 12;
                continue;
            }
        }
        const uint64_t e = umin64(to, ((p >> 12) + 1) << 12);  // to the end of p's superblock
        const uint64_t r = w_first_geq(S, R, p, e, M, val);
        if (r < e) return r;
        p = e;
    }
    return to;
}

// RAM next(s) for the whole warp, the scan skipping superblocks (equals next_ram)
__device__ uint64_t w_next_ram_far(const SumView& S, const RawView& R, const Prm& P, uint64_t fhi, uint64_t s) {
    if (fhi - s <= P.w) return fhi;
    const uint64_t limit = umin64(fhi, s + P.mx);
    const uint64_t t = s + P.w;
    const uint32_t M = w_range_max(S, R, s, t);
    const uint64_t j0 = umax64(t, s + P.mn - 1);
    if (j0 >= limit) return limit;
    if (M == 0) return j0 + 1;
    uint32_t val;
    const uint64_t j = w_first_geq_far(S, R, j0, limit, M, &val);
    return j < limit ? j + 1 : limit;
}

// advance_far() for the whole warp: k steps of stride d, then e (quiet runs and
// runs of forced cuts in one call), the RAM scan skipping superblocks
template <int RULE>
__device__ uint64_t w_advance_far(const SumView& S, const RawView& R, const Prm& P, uint64_t flo, uint64_t fhi,
                                  uint64_t s, uint64_t stop, uint32_t* k, uint64_t* d) {
    if (RULE == RULE_RAM) {
        const uint64_t w = P.w, st = w + 1;
        if (P.mn <= st && s + w < fhi && S.m(s >> 6) == 0 && S.m((s + w - 1) >> 6) == 0) {
            const uint64_t kstop = (stop - 1 - s) / st + 1;
            const uint64_t kfhi = (fhi - 1 - s - w) / st + 1;
            const uint64_t kmax = kstop < kfhi ? kstop : kfhi;
            const uint64_t z = w_first_nonzero(S, R, s, s + (kmax - 1) * st + w + 1);
            const uint64_t kz = z > s + w ? (z - 1 - s - w) / st + 1 : 0;
            const uint64_t kk = kz < kmax ? kz : kmax;
            if (kk >= 2) {
                *k = (uint32_t)kk;
                *d = st;
                return s + kk * st;
            }
        }
        const uint64_t e = w_next_ram_far(S, R, P, fhi, s);
        *k = 1;
        *d = e - s;
        return e;
    }
    return w_advance<RULE>(S, R, P, flo, fhi, s, stop, k, d);
}

// F(y) by stepping the chain (cand_next_t) with every step shared by the
// warp's lanes (warp_rules.cuh): the same landing and count. Quiet runs and
// runs of forced cuts are crossed in one step; their cuts are not candidates.
template <int RULE>
__device__ uint64_t w_cand_next(const SumView& S, const RawView& R, const Prm& P, uint64_t lo, uint64_t hi,
                                uint64_t y, uint32_t* n) {
    uint64_t s = y;
    uint32_t c = 0;
    for (;;) {
        uint64_t e;
        if (RULE == RULE_RAM || RULE == RULE_AE) {
            const uint64_t w = P.w, st = w + 1;
            if (P.mn <= st && s + w < hi && S.m(s >> 6) == 0 && S.m((s + w - 1) >> 6) == 0) {
                // a zero run: cuts every w + 1 bytes, none of them a candidate
                const uint64_t kmax = (hi - 1 - s - w) / st + 1;
                const uint64_t z = w_first_nonzero(S, R, s, s + (kmax - 1) * st + w + 1);
                const uint64_t kz = z > s + w ? (z - 1 - s - w) / st + 1 : 0;
                const uint64_t kk = kz < kmax ? kz : kmax;
                if (kk >= 1) {
                    c += (uint32_t)kk;
                    s += kk * st;
                    if (s >= hi) {
                        *n = c;
                        return hi;
                    }
                    continue;
                }
            }
            e = RULE == RULE_RAM ? w_next_ram_far(S, R, P, hi, s) : w_next_ae(S, R, P, hi, s);
            c++;
        } else {
            uint32_t k;
            uint64_t d;
            e = w_advance<RULE>(S, R, P, lo, hi, s, hi, &k, &d);
            c += k;
        }
        if (e >= hi || e <= s) {  // (e <= s cannot happen: every chunk holds a byte)
            *n = c;
            return hi;
        }
        if (w_is_cand<RULE>(S, R, P, lo, hi, e)) {
            *n = c;
            return e;
        }
        s = e;
    }
}

// window maximum over bytes [a, b): blocks [sb0, sb0 + sn) staged (sm) with
// their running maxima inside superblocks (spr, ssf); ranges outside the
// staged blocks go to the global summaries
struct WMaxStaged {
    const uint8_t* sm;   // block maxima of blocks [sb0, sb0 + sn)
    const uint8_t* spr;  // their running maxima inside superblocks, or null
    const uint8_t* ssf;
    uint64_t sb0, sn;
    const SumView* S;
    const PreSuf* T;
    const RawView* R;
    __device__ uint32_t whole(uint64_t fb, uint64_t lb) const {  // blocks [fb, lb), staged
        if (spr) {
            const uint64_t q0 = fb >> 6, q1 = (lb - 1) >> 6;
            if (q0 == q1) {
                if ((fb & 63) == 0) return spr[lb - 1 - sb0];
                if ((lb & 63) == 0) return ssf[fb - sb0];
            } else {
                uint32_t M = ssf[fb - sb0];
                const uint32_t t = spr[lb - 1 - sb0];
                if (t > M) M = t;
                for (uint64_t q = q0 + 1; q < q1 && M < 255; q++) {
                    const uint32_t u = S->sup[q];
                    if (u > M) M = u;
                }
                return M;
            }
        }
        uint32_t M = 0;
        for (uint64_t x = fb; x < lb; x++) {
            const uint32_t t = sm[x - sb0];
            if (t > M) M = t;
        }
        return M;
    }
    __device__ uint32_t operator()(uint64_t a, uint64_t b) const {
        const uint64_t ba = a >> 6, bl = (b - 1) >> 6;
        if (ba < sb0 || bl >= sb0 + sn) return range_max_t(*S, *T, *R, a, b);
        if (ba == bl) {
            const uint32_t m = sm[ba - sb0];
            if (m == 0 || ((a & 63) == 0 && (b & 63) == 0)) return m;
            return raw_max(*R, a, b);
        }
        const uint64_t fb = (a + 63) >> 6, lb = b >> 6;
        uint32_t M = fb < lb ? whole(fb, lb) : 0;
        if (M == 255) return 255;
        if ((a & 63) && sm[ba - sb0] > M) {
            const uint32_t h = raw_max(*R, a, (ba + 1) << 6);
            if (h > M) M = h;
        }
        if ((b & 63) && sm[bl - sb0] > M) {
            const uint32_t t = raw_max(*R, bl << 6, b);
            if (t > M) M = t;
        }
        return M;
    }
};

// copy n words / bytes from global (16-byte aligned) to shared memory
__device__ __forceinline__ void g_copy_u32(uint32_t* dst, const uint32_t* src, uint32_t n, int tid, int nt) {
    const uint32_t nv = n / 4;
    for (uint32_t q = (uint32_t)tid; q < nv; q += (uint32_t)nt)
        reinterpret_cast<uint4*>(dst)[q] = reinterpret_cast<const uint4*>(src)[q];
    for (uint32_t i = nv * 4 + (uint32_t)tid; i < n; i += (uint32_t)nt) dst[i] = src[i];
}
__device__ __forceinline__ void g_copy_u8(uint8_t* dst, const uint8_t* src, uint32_t n, int tid, int nt) {
    const uint32_t nv = n / 16;
    for (uint32_t q = (uint32_t)tid; q < nv; q += (uint32_t)nt)
        reinterpret_cast<uint4*>(dst)[q] = reinterpret_cast<const uint4*>(src)[q];
    for (uint32_t i = nv * 16 + (uint32_t)tid; i < n; i += (uint32_t)nt) dst[i] = src[i];
}

template <int RULE, int GL_THREADS>
__global__ void __launch_bounds__(GL_THREADS, 512 / GL_THREADS) k_glocal(GraphLaunch A) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t cap = A.cap;
    uint32_t* lpos = reinterpret_cast<uint32_t*>(smem);  // own then next segment's candidates - segment start
    uint32_t* J = lpos + 2 * cap;                         // own index the jump leads to, or GL_EXIT
    uint32_t* C = J + cap;                                // chunk ends covered by the jump
    uint32_t* X = C + cap;                                // exit id (valid once J is GL_EXIT)
    uint8_t* lval = reinterpret_cast<uint8_t*>(X + cap);  // the candidates' bytes
    uint8_t* lgm = lval + 2 * cap;                        // their maxima per group of 32
    uint8_t* sm = smem + gl_stage_off(cap);               // staged block maxima
    uint8_t* spr = sm + A.win;                            // running maxima inside superblocks (staged)
    uint8_t* ssf = sm + 2 * A.win;
    uint32_t* pq = reinterpret_cast<uint32_t*>(smem + gl_queue_off(RULE, cap, A.win));  // F by stepping
    __shared__ uint32_t s_seg, s_np;
    const int tid = threadIdx.x;
    const Prm P{A.w, A.mn, A.mx};
    const RawView R{A.base, A.inv};
    const SumView S{A.smax, A.sarg, nullptr, nullptr, 0, 0, A.ssup};
    const PreSuf T{A.spre, A.ssuf};
    const uint64_t nblk_all = ((A.hi + 63) >> 6) + 16;
    unsigned long long* st = A.stats;  // counters (testing only)
    for (;;) {
        long long t0 = st ? clock64() : 0;
        if (tid == 0) {
            s_seg = (uint32_t)atomicAdd(A.ticket, 1ull);
            s_np = 0;
        }
        __syncthreads();
        const uint32_t seg = s_seg;
        if (seg >= A.nseg) break;
        const uint64_t a = g_seg_lo(A, seg), b = g_seg_hi(A, seg);
        const uint32_t n = g_slot_n(A, seg);
        const bool has_next = seg + 1 < A.nseg;
        const uint32_t nla = has_next ? g_slot_n(A, seg + 1) : 0u;
        const uint64_t base = (uint64_t)seg * cap;
        // lists: slots start at multiples of 16 entries, so 16-byte loads
        g_copy_u32(lpos, A.cpos + base, n, tid, GL_THREADS);
        g_copy_u8(lval, A.cval + base, n, tid, GL_THREADS);
        if (nla) {
            const uint32_t shift = (uint32_t)(b - a);
            for (uint32_t i = tid; i < nla; i += GL_THREADS) {
                lpos[n + i] = shift + A.cpos[base + cap + i];
                lval[n + i] = A.cval[base + cap + i];
            }
        }
        // the list is complete up to (and including) this position
        uint64_t cover;
        if (A.cnum[seg] > cap) {
            cover = n ? a + A.cpos[base + n - 1] : a;
        } else if (!has_next) {
            cover = A.hi;
        } else if (A.cnum[seg + 1] > cap) {
            cover = nla ? b + A.cpos[base + cap + nla - 1] : b;
        } else {
            cover = g_seg_hi(A, seg + 1) - 1;
        }
        // stage the block maxima (and the window table, if any) from 2w + 128
        // bytes before the segment up to the end of the next one
        uint64_t sb0 = 0, sn = 0;
        if (RULE != RULE_MAXP) {
            const uint64_t back = 2ull * A.w + 128;
            const uint64_t from = a > A.lo + back ? a - back : A.lo;
            sb0 = (from >> 6) & ~15ull;
            const uint64_t upto = ((has_next ? g_seg_hi(A, seg + 1) : b) + 63) >> 6;
            sn = (upto + 1 - sb0 + 15) & ~15ull;
            if (sn > A.win) sn = A.win;
            const uint64_t lim = nblk_all & ~15ull;
            if (sb0 + sn > lim) sn = lim > sb0 ? lim - sb0 : 0;
            for (uint32_t q = tid; q < sn / 16; q += GL_THREADS) {
                reinterpret_cast<uint4*>(sm)[q] = reinterpret_cast<const uint4*>(A.smax + sb0)[q];
                if (A.spre) {
                    reinterpret_cast<uint4*>(spr)[q] = reinterpret_cast<const uint4*>(A.spre + sb0)[q];
                    reinterpret_cast<uint4*>(ssf)[q] = reinterpret_cast<const uint4*>(A.ssuf + sb0)[q];
                }
            }
        }
        __syncthreads();
        long long t1 = st ? clock64() : 0;
        for (uint32_t g = tid; g < (n + nla + 31) / 32; g += GL_THREADS) {
            uint32_t m = 0;
            for (uint32_t i = g * 32; i < g * 32 + 32 && i < n + nla; i++) m = lval[i] > m ? lval[i] : m;
            lgm[g] = (uint8_t)m;
        }
        __syncthreads();
        const WMaxStaged wm{sm, A.spre ? spr : nullptr, ssf, sb0, sn, &S, &T, &R};
        const CandList L{lpos, lval, n + nla, a, cover, lgm};
        // F from the lists; the candidates the lists cannot decide are queued
        for (uint32_t i = tid; i < n; i += GL_THREADS) {
            const uint64_t y = a + lpos[i];
            uint32_t cnt;
            const uint32_t k = list_next<RULE>(L, wm, R, P, A.flo, A.hi, y, &cnt);
            if (k == LIST_GENERIC) {
                J[i] = GL_PEND;
                pq[atomicAdd(&s_np, 1u)] = i;
                continue;
            }
            uint32_t ft, jj = GL_EXIT;
            if (k < n) {
                ft = seg * cap + k;
                jj = k;
            } else {
                ft = (seg + 1) * cap + (k - n);
            }
            A.cft[base + i] = ft;
            A.csc[base + i] = cnt;
            J[i] = jj;
            C[i] = cnt;
            X[i] = ft;
        }
        __syncthreads();
        {
            // the queued candidates, one warp each: F by stepping the chain
            const uint32_t np = s_np;
            const int lane = tid & 31;
            for (uint32_t q = (uint32_t)(tid >> 5); q < np; q += GL_THREADS / 32) {
                const uint32_t i = pq[q];
                const uint64_t y = a + lpos[i];
                uint32_t c = 1, ft, jj = GL_EXIT;
                const long long tg = st ? clock64() : 0;
                const uint64_t e = w_cand_next<RULE>(S, R, P, A.flo, A.hi, y, &c);
                if (lane != 0) continue;
                if (st) {
                    const unsigned long long dt = (unsigned long long)(clock64() - tg);
                    atomicAdd(&st[GST_GENERIC], 1ull);
                    atomicAdd(&st[GST_CYC_GENERIC], dt);
                    atomicMax(&st[GST_MAX_GENERIC], dt);
                }
                if (e >= A.hi) {
                    ft = GID_END;
                } else if (e <= cover) {
                    const uint32_t k2 = list_lower_bound(L, e);
                    if (k2 < n + nla && a + lpos[k2] == e) {
                        if (k2 < n) {
                            ft = seg * cap + k2;
                            jj = k2;
                        } else {
                            ft = (seg + 1) * cap + (k2 - n);
                        }
                    } else {
                        ft = GID_SLOW;
                        g_fail(A, y);  // every candidate up to `cover` is listed
                    }
                } else {
                    ft = g_find(A, g_seg_of(A, e), e);
                    if (ft < GID_NONE && A.cfar[ft] == 0) {
                        // a far landing: list it for the unit tables
                        const unsigned long long at = atomicAdd(&A.ticket[1], 1ull);
                        if (at < A.far_cap) {
                            A.far_list[at] = ft;
                            A.cfar[ft] = 1;
                        }
                    }
                }
                A.cft[base + i] = ft;
                A.csc[base + i] = c;
                J[i] = jj;
                C[i] = c;
                X[i] = ft;
            }
        }
        __syncthreads();
        long long t2 = st ? clock64() : 0;
        // pointer jumping: after round r each J covers 2^r F steps or has left
        uint32_t rounds = 0;
        for (;;) {
            uint32_t nj[GL_PER], nc[GL_PER], nx[GL_PER];
            int act = 0;
#pragma unroll
            for (int r = 0; r < GL_PER; r++) {
                const uint32_t i = (uint32_t)tid + (uint32_t)r * GL_THREADS;
                nj[r] = GL_EXIT;
                if (i < n && J[i] != GL_EXIT) {
                    const uint32_t j = J[i];
                    nj[r] = J[j];
                    nc[r] = C[i] + C[j];
                    nx[r] = X[j];
                    act |= 1 << r;
                }
            }
            if (!__syncthreads_or(act)) break;
            rounds++;
#pragma unroll
            for (int r = 0; r < GL_PER; r++) {
                if (act & (1 << r)) {
                    const uint32_t i = (uint32_t)tid + (uint32_t)r * GL_THREADS;
                    J[i] = nj[r];
                    C[i] = nc[r];
                    X[i] = nx[r];
                }
            }
            __syncthreads();
        }
        for (uint32_t i = tid; i < n; i += GL_THREADS) A.cex[base + i] = ((unsigned long long)C[i] << 32) | X[i];
        if (st && tid == 0) {
            const long long t3 = clock64();
            atomicAdd(&st[GST_SEGMENTS], 1ull);
            atomicAdd(&st[GST_CANDS], (unsigned long long)n);
            atomicAdd(&st[GST_CYC_STAGE], (unsigned long long)(t1 - t0));
            atomicAdd(&st[GST_CYC_F], (unsigned long long)(t2 - t1));
            atomicAdd(&st[GST_CYC_JUMP], (unsigned long long)(t3 - t2));
            atomicAdd(&st[GST_ROUNDS], (unsigned long long)rounds);
            atomicMax(&st[GST_MAX_SEG], (unsigned long long)(t3 - t0));
            atomicMax(&st[GST_MAX_STAGE], (unsigned long long)(t1 - t0));
            atomicMax(&st[GST_MAX_F], (unsigned long long)(t2 - t1));
            atomicMax(&st[GST_MAX_JUMP], (unsigned long long)(t3 - t2));
            atomicMax(&st[GST_MAX_SEG_AT], ((unsigned long long)(t3 - t0) << 24) | seg);
        }
        __syncthreads();  // shared arrays (and s_seg) are reused by the next segment
    }
}

// ---- staged exit tables for the chase ------------------------------------------------
//
// The chase kernels (k_gunit, k_gtop, k_gdesc) follow chains hop by hop, each
// hop a load that depends on the previous one. A CTA first copies the table
// entries its walks can read (the exits of a unit's segments, or the unit
// exits of every unit's first segment) into shared memory with coalesced
// loads, so that the hops themselves read shared memory. Tables that do not
// fit are read from global memory as before.

constexpr int GU_THREADS = 512;
constexpr uint32_t GU_MAXP = 256;                  // parts (segments or units) a staged table spans
constexpr uint32_t GU_ENTRIES = 24576;             // staged entries (8 bytes each)
int graph_chase_smem() { return (int)(GU_ENTRIES * 8u); }

struct StagedTab {
    const unsigned long long* ent;  // entries of part j at ent[off[j]], part j = segment k0 + j * step
    const uint32_t* off;
    uint32_t k0, step, parts;
    bool ok;
};

// Copy the first g_slot_n(k) entries (rounded up to an even count: 16-byte
// copies) of src[k * cap ...] for the segments k = k0 + j * step (j < parts)
// into ent, with the bulk-copy engine (one copy per part, completed on the
// mbarrier `bar`; *phase counts its uses). False (nothing staged) if they do
// not fit or the copies do not complete in time.
__device__ bool g_stage(const GraphLaunch& A, const unsigned long long* src, uint32_t k0, uint32_t step,
                        uint32_t parts, unsigned long long* ent, uint32_t* off, uint64_t* bar, uint32_t* phase) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (parts > GU_MAXP) return false;
    for (uint32_t j = tid; j < parts; j += nt) off[j + 1] = (g_slot_n(A, k0 + j * step) + 1u) & ~1u;
    __syncthreads();
    if (tid == 0) {
        off[0] = 0;
        for (uint32_t j = 0; j < parts; j++) off[j + 1] += off[j];
    }
    __syncthreads();
    const uint32_t tot = off[parts];
    if (tot > GU_ENTRIES) return false;
    if (tot == 0) return true;
    if (tid == 0) {
        // the buffer was last read by ordinary loads: order them before the copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, tot * 8u);
        for (uint32_t j = 0; j < parts; j++) {
            const uint32_t n = off[j + 1] - off[j];
            if (n) bulk_g2s(ent + off[j], src + (uint64_t)(k0 + j * step) * A.cap, n * 8u, bar);
        }
    }
    const uint32_t par = *phase & 1u;
    *phase += 1;
    bool ok = mbar_wait_bounded(bar, par, A.timeout_ns);
    if (!ok) {
        // flag it, and let the copies in flight land before the buffer is reused
        if (tid == 0) atomicOr(&A.ctrl->err, ERR_TIMEOUT);
        mbar_wait_bounded(bar, par, A.timeout_ns);
    }
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// one mbarrier for g_stage, initialised by the CTA
__device__ __forceinline__ void g_stage_init(uint64_t* bar) {
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
}

// the table entry of candidate id: staged if id's segment is a staged part
__device__ __forceinline__ unsigned long long g_tab(const GraphLaunch& A, const StagedTab& T,
                                                    const unsigned long long* src, uint32_t id) {
    const uint32_t k = id / A.cap;
    if (T.ok && k >= T.k0) {
        const uint32_t d = k - T.k0;
        if (d % T.step == 0 && d / T.step < T.parts) return T.ent[T.off[d / T.step] + (id - k * A.cap)];
    }
    return src[id];
}

// ---- k_gunit: exits of each unit's first segment past the unit ----------------

template <int RULE>
__device__ __forceinline__ unsigned long long g_unit_exit(const GraphLaunch& A, const StagedTab& T, uint32_t id) {
    const uint32_t kend0 = (id / A.cap / A.G + 1) * A.G;
    const uint32_t kend = kend0 < A.nseg ? kend0 : A.nseg;
    unsigned long long acc = 0;
    for (uint32_t guard = 0; id < GID_NONE && id / A.cap < kend; guard++) {
        unsigned long long v = g_tab(A, T, A.cex, id);
        if ((uint32_t)v == GID_SLOW) v = g_slow_hop<RULE>(A, id);
        if ((uint32_t)v <= id || guard > A.G) {  // ids only grow along a chain, one segment at least
            g_fail(A, id);
            id = GID_END;
            break;
        }
        acc += v >> 32;
        id = (uint32_t)v;
    }
    return (acc << 32) | id;
}

template <int RULE>
__global__ void __launch_bounds__(GU_THREADS) k_gunit(GraphLaunch A) {
    extern __shared__ __align__(16) unsigned long long gu_ent[];
    __shared__ uint32_t gu_off[GU_MAXP + 1];
    __shared__ uint64_t gu_bar;
    g_stage_init(&gu_bar);
    uint32_t phase = 0;
    // (a) every candidate of each unit's first segment, over the unit's staged exits
    for (uint32_t u = blockIdx.x; u < A.nunit; u += gridDim.x) {
        const uint32_t k0 = u * A.G;
        const uint32_t parts = (k0 + A.G < A.nseg ? k0 + A.G : A.nseg) - k0;
        StagedTab T{gu_ent, gu_off, k0, 1, parts, false};
        T.ok = g_stage(A, A.cex, k0, 1, parts, gu_ent, gu_off, &gu_bar, &phase);
        const uint32_t n0 = g_slot_n(A, k0);
        for (uint32_t i = threadIdx.x; i < n0; i += blockDim.x) {
            const uint32_t id = k0 * A.cap + i;
            A.cux[id] = g_unit_exit<RULE>(A, T, id);
        }
        __syncthreads();  // the staged table is replaced by the next unit's
    }
    // (b) the far landings (a chain entering a unit past its first segment)
    const StagedTab none{nullptr, nullptr, 0, 1, 0, false};
    const unsigned long long nf0 = A.ticket[1];
    const uint32_t nf = nf0 < A.far_cap ? (uint32_t)nf0 : A.far_cap;
    for (uint32_t f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        const uint32_t id = A.far_list[f];
        if ((id / A.cap) % A.G != 0) A.cux[id] = g_unit_exit<RULE>(A, none, id);
    }
}

// ---- k_gtop: the true chain over the units (or the segments) ----------------------

template <int RULE>
__global__ void __launch_bounds__(GU_THREADS) k_gtop(GraphLaunch A) {
    extern __shared__ __align__(16) unsigned long long gu_ent[];
    __shared__ uint32_t gu_off[GU_MAXP + 1];
    __shared__ uint64_t gu_bar;
    g_stage_init(&gu_bar);
    uint32_t phase = 0;
    // the unit exits of every unit's first segment, staged
    StagedTab T{gu_ent, gu_off, 0, A.G, A.nunit, false};
    if (A.nunit > 1) T.ok = g_stage(A, A.cux, 0, A.G, A.nunit, gu_ent, gu_off, &gu_bar, &phase);
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t id = 0;  // segment 0, slot 0: the first byte
    unsigned long long off = 0;
    // every hop leads to a larger id (a later segment), so the loops below end
    // after at most nseg hops; the checks only guard against a broken table
    uint32_t hops = 0;
    auto next = [&](unsigned long long v) {
        if ((uint32_t)v <= id || ++hops > 2 * A.nseg + 2) {
            g_fail(A, id);
            id = GID_NONE;
            return;
        }
        off += v >> 32;
        id = (uint32_t)v;
    };
    if (A.nunit <= 1) {
        while (id < GID_NONE) {
            const uint32_t k = id / A.cap;
            A.sent[k] = id;
            A.soff[k] = off;
            next(g_hop<RULE>(A, id));
        }
    } else {
        while (id < GID_NONE) {
            const uint32_t k = id / A.cap, u = k / A.G;
            A.uent[u] = id;
            A.uoff[u] = off;
            if (k == u * A.G) {
                next(g_tab(A, T, A.cux, id));
                continue;
            }
            // both loads at once: the flag decides which one the hop uses
            const unsigned long long vu = A.cux[id];
            const uint8_t far = A.cfar[id];
            if (far) {
                next(vu);
            } else {
                const uint32_t kend = (u + 1) * A.G;
                while (id < GID_NONE && id / A.cap < kend) next(g_hop<RULE>(A, id));
            }
        }
    }
    if (id != GID_END) g_fail(A, 0xFFFFFFFFull);
    A.ctrl->total = off;
    if (A.d_count) *A.d_count = off;
}

// ---- k_gdesc: each unit's segments ---------------------------------------------------

template <int RULE>
__global__ void __launch_bounds__(GU_THREADS) k_gdesc(GraphLaunch A) {
    extern __shared__ __align__(16) unsigned long long gu_ent[];
    __shared__ uint32_t gu_off[GU_MAXP + 1];
    __shared__ uint64_t gu_bar;
    g_stage_init(&gu_bar);
    uint32_t phase = 0;
    for (uint32_t u = blockIdx.x; u < A.nunit; u += gridDim.x) {
        uint32_t id = A.uent[u];
        if (id >= GID_NONE) continue;  // (uniform over the CTA)
        const uint32_t k0 = u * A.G;
        const uint32_t parts = (k0 + A.G < A.nseg ? k0 + A.G : A.nseg) - k0;
        StagedTab T{gu_ent, gu_off, k0, 1, parts, false};
        T.ok = g_stage(A, A.cex, k0, 1, parts, gu_ent, gu_off, &gu_bar, &phase);
        if (threadIdx.x == 0) {
            unsigned long long off = A.uoff[u];
            const uint32_t kend = (u + 1) * A.G;
            for (uint32_t hops = 0; id < GID_NONE && id / A.cap < kend; hops++) {
                const uint32_t k = id / A.cap;
                A.sent[k] = id;
                A.soff[k] = off;
                unsigned long long v = g_tab(A, T, A.cex, id);
                if ((uint32_t)v == GID_SLOW) v = g_slow_hop<RULE>(A, id);
                if ((uint32_t)v <= id || hops > A.G) {
                    g_fail(A, id);
                    break;
                }
                off += v >> 32;
                id = (uint32_t)v;
            }
        }
        __syncthreads();  // the staged table is replaced by the next unit's
    }
}

// ---- k_gemit: boundaries of each segment's part of the true chain ------------------
//
// The segment's F targets, step counts and positions are staged in shared
// memory (coalesced), then one thread replays the true chain from the
// segment's entry, candidate after candidate, into a shared buffer that the
// CTA stores together. Where F took more than one step (forced cuts, quiet
// runs) or a candidate has no slot, the thread steps the chain itself.

constexpr int GE_THREADS = 128;

int graph_emit_smem(uint32_t cap) { return (int)(((12u * cap + 15u) & ~15u) + 8u * GE_BUF); }

template <int RULE>
__global__ void __launch_bounds__(GE_THREADS) k_gemit(GraphLaunch A) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t cap = A.cap;
    uint32_t* sft = reinterpret_cast<uint32_t*>(smem);
    uint32_t* ssc = sft + cap;
    uint32_t* spos = ssc + cap;
    unsigned long long* buf = reinterpret_cast<unsigned long long*>(smem + ((12u * cap + 15u) & ~15u));
    __shared__ uint32_t s_held;
    __shared__ int s_done;
    __shared__ unsigned long long s_nb;
    const int tid = threadIdx.x;
    const Prm P{A.w, A.mn, A.mx};
    const RawView R{A.base, A.inv};
    const SumView S{A.smax, A.sarg, nullptr, nullptr, 0, 0, A.ssup};
    for (uint32_t seg = blockIdx.x; seg < A.nseg; seg += gridDim.x) {
        const uint32_t id0 = A.sent[seg];
        if (id0 >= GID_NONE) continue;
        const uint64_t a = g_seg_lo(A, seg);
        const uint32_t n = g_slot_n(A, seg);
        const uint64_t base = (uint64_t)seg * cap;
        g_copy_u32(sft, A.cft + base, n, tid, GE_THREADS);
        g_copy_u32(ssc, A.csc + base, n, tid, GE_THREADS);
        g_copy_u32(spos, A.cpos + base, n, tid, GE_THREADS);
        __syncthreads();
        const unsigned long long off0 = A.soff[seg];
        if (tid == 0) s_nb = 0;
        // walk state (thread 0): current chunk start y and its candidate index
        // in this segment (or ~0u: a position without a slot)
        uint64_t y = a + spos[id0 - base];
        uint32_t cur = id0 - (uint32_t)base;
        for (;;) {
            if (tid < 32) {  // warp 0 walks (every lane the same state); lane 0 fills the buffer
                const int lane = tid;
                uint32_t held = 0;
                unsigned long long nb = s_nb;  // boundaries stored so far
                bool done = false;
                while (!done && held < GE_BUF - 64) {
                    const uint32_t ft = cur != ~0u ? sft[cur] : GID_SLOW;
                    uint64_t e;
                    uint32_t nxt;
                    if (ft != GID_SLOW && ssc[cur] == 1) {
                        if (ft == GID_END) e = A.hi;
                        else if (ft >= (uint32_t)base && ft - (uint32_t)base < n) e = a + spos[ft - (uint32_t)base];
                        else e = g_pos(A, ft);
                        if (lane == 0) buf[held] = e - A.lo;
                        held++;
                        nxt = ft;
                    } else {
                        // step the chain: every end up to the next candidate
                        uint64_t s2 = y;
                        for (;;) {
                            uint32_t k;
                            uint64_t d;
                            const uint64_t e2 = w_advance_far<RULE>(S, R, P, A.flo, A.hi, s2, A.hi, &k, &d);
                            for (uint32_t t = 1; t <= k; t++) {
                                if (lane == 0) buf[held] = s2 + t * d - A.lo;
                                held++;
                                if (held == GE_BUF) {
                                    // rare (long quiet or forced runs): the warp stores the buffer
                                    __syncwarp();
                                    for (uint32_t q = (uint32_t)lane; q < held; q += 32)
                                        if (off0 + nb + q < A.capacity) A.out[off0 + nb + q] = buf[q];
                                    __syncwarp();
                                    nb += held;
                                    held = 0;
                                }
                            }
                            if (e2 <= s2) {  // (cannot happen: every chunk holds a byte)
                                g_fail(A, seg);
                                s2 = A.hi;
                                break;
                            }
                            s2 = e2;
                            if (e2 >= A.hi || w_is_cand<RULE>(S, R, P, A.flo, A.hi, e2)) break;
                        }
                        e = s2;
                        if (ft != GID_SLOW) nxt = ft;
                        else if (e >= A.hi) nxt = GID_END;
                        else nxt = g_find(A, g_seg_of(A, e), e);
                    }
                    if (e <= y) {  // the chain only moves forward, so the walk ends
                        g_fail(A, seg);
                        done = true;
                    } else if (e >= A.hi) {
                        done = true;
                    } else if (g_seg_of(A, e) != seg && nxt != GID_SLOW) {
                        done = true;  // the first candidate past the segment: its segment goes on
                    } else {
                        y = e;
                        cur = (nxt < GID_NONE && nxt >= (uint32_t)base && nxt - (uint32_t)base < n)
                                  ? nxt - (uint32_t)base
                                  : ~0u;
                    }
                }
                if (lane == 0) {
                    s_nb = nb;
                    s_held = held;
                    s_done = done ? 1 : 0;
                }
            }
            __syncthreads();
            const uint32_t held = s_held;
            const bool done = s_done != 0;
            const unsigned long long nb = s_nb;
            for (uint32_t q = (uint32_t)tid; q < held; q += GE_THREADS) {
                const unsigned long long o = off0 + nb + q;
                if (o < A.capacity) A.out[o] = buf[q];
            }
            __syncthreads();
            if (tid == 0) s_nb = nb + held;
            __syncthreads();
            if (done) break;
        }
        if (tid == 0) {
            const unsigned long long v = A.cex[id0];
            if ((uint32_t)v != GID_SLOW && (v >> 32) != s_nb) g_fail(A, seg);
        }
        __syncthreads();  // shared arrays are reused by the next segment
    }
}

// ---- launcher ---------------------------------------------------------------------------

template <int RULE>
static int g_allow_smem() {
    return launch_memo(400 + RULE, 0, [](uint32_t) {
        int e = allow_max_smem(k_glocal<RULE, 512>);
        if (e == 0) e = allow_max_smem(k_glocal<RULE, 256>);
        if (e == 0) e = allow_max_smem(k_gemit<RULE>);
        if (e == 0) e = allow_max_smem(k_gunit<RULE>);
        if (e == 0) e = allow_max_smem(k_gtop<RULE>);
        if (e == 0) e = allow_max_smem(k_gdesc<RULE>);
        return e;
    });
}

template <int RULE>
static int g_occ_local(uint32_t key) {
    g_allow_smem<RULE>();
    return launch_memo(410 + RULE, key, [](uint32_t kk) {
        const uint32_t cap = kk >> 16, win = (kk & 0xFFFFu) * 16;
        int n = 0;
        if (cap <= 2048)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_glocal<RULE, 256>, 256,
                                                          graph_local_smem(RULE, cap, win));
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_glocal<RULE, 512>, 512,
                                                          graph_local_smem(RULE, cap, win));
        return n > 0 ? n : 1;
    });
}

int graph_local_blocks_per_sm(int rule, uint32_t cap, uint32_t win) {
    const uint32_t key = (cap << 16) | (win / 16);
    switch (rule) {
    case RULE_RAM: return g_occ_local<RULE_RAM>(key);
    case RULE_AE: return g_occ_local<RULE_AE>(key);
    default: return g_occ_local<RULE_MAXP>(key);
    }
}

template <int RULE>
static cudaError_t launch_graph_rule(const GraphLaunch& a, const GraphGrids& g, cudaStream_t st, int* launches,
                                     cudaEvent_t ev_mid) {
    const int set = g_allow_smem<RULE>();
    if (set != (int)cudaSuccess) return (cudaError_t)set;
    k_gcand<RULE><<<g.cand, GC_THREADS, 0, st>>>(a);
    if (a.cap <= 2048)
        k_glocal<RULE, 256><<<g.local, 256, graph_local_smem(RULE, a.cap, a.win), st>>>(a);
    else
        k_glocal<RULE, 512><<<g.local, 512, graph_local_smem(RULE, a.cap, a.win), st>>>(a);
    if (ev_mid) cudaEventRecord(ev_mid, st);
    int n = 4;
    const int csm = graph_chase_smem();
    if (a.nunit > 1) {
        k_gunit<RULE><<<g.unit, GU_THREADS, csm, st>>>(a);
        n++;
    }
    k_gtop<RULE><<<1, GU_THREADS, csm, st>>>(a);
    if (a.nunit > 1) {
        k_gdesc<RULE><<<g.unit, GU_THREADS, csm, st>>>(a);
        n++;
    }
    k_gemit<RULE><<<g.emit, GE_THREADS, graph_emit_smem(a.cap), st>>>(a);
    *launches += n;
    return cudaGetLastError();
}

cudaError_t launch_graph(const GraphLaunch& a, int rule, const GraphGrids& g, cudaStream_t st, int* launches,
                         cudaEvent_t ev_mid) {
    switch (rule) {
    case RULE_RAM: return launch_graph_rule<RULE_RAM>(a, g, st, launches, ev_mid);
    case RULE_AE: return launch_graph_rule<RULE_AE>(a, g, st, launches, ev_mid);
    case RULE_MAXP: return launch_graph_rule<RULE_MAXP>(a, g, st, launches, ev_mid);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace cdc
