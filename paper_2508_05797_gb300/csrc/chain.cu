// chain.cu -- stage 2: the chunk chain, in parallel and bit-exact.
//
// Each chunk starts where the previous one ended (Section 3.3: every
// algorithm is a loop over one chunk at a time), so the chunk starts form a
// single chain s_{i+1} = next(s_i). Chains started at different offsets join
// where their cuts coincide, but on random or text-like bytes that can take
// hundreds of kilobytes (the gap between two chains moves like a random
// walk), and inside runs of zeros -- or MAXP stretches without a target --
// they never join at all. The stage therefore splits the input into
// segments and describes each segment by a transfer table over many chains:
//
//  k_spec    (one persistent CTA of NW warps per segment at a time)
//    * Segment bounds: nominal bounds every `seg` bytes are moved forward
//      out of quiet regions (zero superblocks for RAM/AE, target-less runs
//      for MAXP), so that every segment starts where chains join quickly.
//    * Speculate: NL = 32*NW chains from starts spread over the first `span`
//      bytes, first one step per thread per round, then (once few are left)
//      one warp per chain over shared-memory block summaries. Every position a
//      chain steps from goes into a shared-memory hash (a chain that lands on
//      a hashed position has joined another and stops), and every step into
//      the segment's step log.
//  k_stitch  (after all speculation; no waits): for each distinct exit of the
//            nearest non-empty predecessor, a warp follows the chain from that
//            exit until it lands on a hashed position (or ends on a chain's
//            exit). Result: predecessor chain -> (chain, boundaries in segment).
//  k_ures    follows the few exits no chain covers into the next segment.
//  k_compose (one warp per group of A.gs segments, 8..128 chosen per call):
//            composes the group's tables.
//  k_scan    (one warp): carries the true state across the group composites
//            from the start of the data (the first segment of every file is
//            exact), settling entries no table covers by following the chain.
//  k_settle  (one warp per group): carries the state through the group's
//            segments; records each segment's true entry and global offset.
//  k_output  (one warp per segment): replays the true chain from the logs (the
//            stitch walk from its entry, then the speculation log, where the
//            hash names the chain at a position), stepping only where no record
//            covers it, and writes its boundaries at that offset.
// Every wait (a segment on its predecessor's speculation) is bounded.
#include "cdc_device.cuh"
#include "cdc_launch.h"
#include "warp_fast.cuh"

#include <mutex>

namespace cdc {

// ---- per-segment state --------------------------------------------------------

CDC_HD uint32_t stab_enc(uint32_t slot, uint32_t count) { return (slot << 23) | (count & 0x7FFFFFu); }
CDC_HD uint32_t stab_slot(uint32_t e) { return (e >> 23) & 0x7Fu; }
CDC_HD uint32_t stab_count(uint32_t e) { return e & 0x7FFFFFu; }
constexpr uint32_t STAB_UNKNOWN = 0x80000000u;  // count in low bits, exit in unk_exit
constexpr uint32_t STAB_CONST = 0x40000000u;    // all entries identical (first segment of a file)

constexpr int NU = 8;  // uncovered positions resolved per segment

struct __align__(128) SegState {
    unsigned long long X[NL];         // chain exits (first position >= seg_hi), ~0 if idle
    unsigned int cnt[NL];             // boundaries of each chain inside the segment
    unsigned int table[NL];           // predecessor chain -> (chain, count)
    unsigned long long unk_exit[NL];  // exit of the followed chain for UNKNOWN entries
    unsigned long long seg_lo, seg_hi, flo, fhi;
    unsigned int geo;                 // bit0 first of file, bit1 last of file, bit2 empty
    unsigned int flagA;               // X, counts, geometry, hash and step log published
    unsigned int log_n;               // records in the step log (> logcap: it overflowed)
    unsigned int ures_n;              // entries of ures_* below
    // positions that reach this segment off every chain (the nearest non-empty
    // predecessor's uncovered exits), each followed here like a stitch walk
    unsigned long long ures_pos[NU];
    unsigned long long ures_exit[NU]; // exit when that walk met no chain either
    unsigned int ures_val[NU];        // table encoding of the walk's result
    // written by k_stitch: where the walk from predecessor exit j is logged
    // (records logcap + sw_first[j] .. + sw_cnt[j]; sw_cnt 0xFFFF: not logged)
    unsigned short sw_first[NL];
    unsigned short sw_cnt[NL];
    // written by k_settle
    unsigned int entry_slot;          // predecessor chain the true path entered by, or NONE
    unsigned long long entry_pos;     // first true position >= seg_lo (or >= seg_hi)
    unsigned long long excl;          // boundaries before this segment
    unsigned int count;               // boundaries inside this segment
    unsigned int fileidx;
};
enum : unsigned int { GEO_FIRST = 1u, GEO_LAST = 2u, GEO_EMPTY = 4u };

size_t seg_state_bytes() { return sizeof(SegState); }

// group composites (k_compose -> k_scan)
struct __align__(128) GroupState {
    unsigned int slot[NL];            // state after the group's last segment, or UNRESOLVED
    unsigned long long count[NL];     // boundaries in the group
    unsigned int entry_slot;          // written by k_scan: state entering the group
    unsigned int pad;
    unsigned long long entry_pos;
    unsigned long long entry_incl;
};
size_t group_state_bytes() { return sizeof(GroupState); }
constexpr uint32_t NONE = 0xFFFFu;
constexpr uint32_t UNRESOLVED = 0xFFFEu;  // composite entry not computable without a walk

// ---- segment geometry ------------------------------------------------------------

struct Geo {
    uint64_t flo, fhi, seg_lo, seg_hi, f;
    bool first;
};

// Move a nominal bound x forward to the first 4 KiB-aligned y whose
// neighbourhood [y - before, y + after) meets no quiet run (a run of at least
// `quiet_run` consecutive quiet superblocks, counted over the whole file).
// The rule depends on y alone, so the result is monotone in x and adjacent
// segments stay contiguous. One forward pass over the superblocks, taken 32
// at a time by the calling warp (every lane returns the same bound): the
// superblock summaries of a batch are loaded at once, and the events of the
// pass -- the window end reached, a quiet run long enough to push y -- are
// found with ballots in the order a single thread would meet them.
__device__ uint64_t adjust_bound(const ChainLaunch& A, uint64_t x, uint64_t flo, uint64_t fhi, int lane) {
    if (A.quiet_run == 0 || x <= flo) return x <= flo ? flo : x;
    if (x >= fhi) return fhi;
    const uint64_t cap = x + A.adj_cap;
    const uint64_t qf = flo >> 12;
    const uint32_t QR = A.quiet_run;
    uint64_t y = x;
    uint64_t q = (y > flo + A.adj_before ? y - A.adj_before : flo) >> 12;
    // length of the quiet run that ends just before q (counted up to QR)
    uint32_t run = 0;
    for (uint64_t r0 = q; run < QR;) {
        const bool qt = r0 > qf + (uint64_t)lane && A.ssup[r0 - 1 - lane] == 0;
        const uint32_t m = __ballot_sync(FULL, qt);
        const uint32_t t = m == FULL ? 32u : (uint32_t)(__ffs((int)~m) - 1);
        run += t;
        if (t < 32) break;
        r0 -= 32;
    }
    if (run > QR) run = QR;
    const uint32_t upto = lane == 31 ? FULL : ((2u << lane) - 1);  // lanes 0..lane
    for (;; q += 32) {
        const uint64_t qq = q + (uint64_t)lane;
        const bool valid = (qq << 12) < fhi;
        const uint32_t qm = __ballot_sync(FULL, valid && A.ssup[qq] == 0);
        uint32_t i = 0;  // batch positions before i are done
        for (;;) {
            const uint32_t from = ~0u << i;
            // the window end, checked first at every position (with the current y)
            const uint32_t tmask = __ballot_sync(FULL, !valid || (qq << 12) >= y + A.adj_after) & from;
            // quiet run ending at each position from i on
            const uint32_t zeros = ~qm & upto & from;
            const uint32_t rj = zeros ? (uint32_t)lane - (31u - (uint32_t)__clz((int)zeros))
                                      : run + (uint32_t)lane - i + 1u;
            const uint32_t gmask = __ballot_sync(FULL, ((qm >> lane) & 1u) && rj >= QR) & from;
            const int ft = tmask ? __ffs((int)tmask) - 1 : 32;
            const int fg = gmask ? __ffs((int)gmask) - 1 : 32;
            if (ft <= fg) {
                if (ft < 32) return y;
                run = __shfl_sync(FULL, rj, 31);  // no event left in this batch
                break;
            }
            uint64_t ny = ((q + (uint64_t)fg + 1) << 12) + A.adj_before;
            ny = (ny + 4095) & ~4095ull;
            if (ny > y) y = ny;
            if (y >= fhi) return fhi;
            if (y >= cap) return cap < fhi ? cap : fhi;
            run = __shfl_sync(FULL, rj, fg);
            i = (uint32_t)fg + 1;
            if (i == 32) break;
        }
    }
}

// Geometry of segment `item`; seg_lo and seg_hi as adjust_bound() gives them.
// Called by whole warps; `bound` selects which bound the warp computes
// (0: seg_lo, 1: seg_hi, 2: both).
__device__ Geo seg_geo(const ChainLaunch& A, uint64_t item, int lane, int bound) {
    Geo g;
    uint64_t flo_l, fhi_l, kin;
    if (A.file_off == nullptr) {
        g.f = 0; flo_l = 0; fhi_l = A.single_len; kin = item;
    } else {
        g.f = A.item_file[item];
        flo_l = A.file_off[g.f];
        fhi_l = A.file_off[g.f + 1];
        kin = item - A.item_off[g.f];
    }
    g.flo = A.lo + flo_l;
    g.fhi = A.lo + fhi_l;
    const uint64_t nlo = g.flo + kin * A.seg, nhi = nlo + A.seg;
    g.first = kin == 0;
    g.seg_lo = g.seg_hi = 0;
    if (bound != 1) g.seg_lo = g.first ? g.flo : adjust_bound(A, nlo, g.flo, g.fhi, lane);
    if (bound != 0) g.seg_hi = nhi >= g.fhi ? g.fhi : adjust_bound(A, nhi, g.flo, g.fhi, lane);
    return g;
}

// ---- shared-memory position hash -----------------------------------------------
// Entries are (key << 32) | value with key = position - seg_lo + 1 and value =
// (chain << 16) | index of the position in that chain. Inserted atomically as
// one 64-bit word, so a chain that finds its position already present learns
// at once which chain got there first.

// Per segment, a position hash of 2^BITS slots (stop inserting beyond FILL
// entries). RAM and AE chains need the 2048-slot table to find their merges;
// MAXP merges within a chunk and takes 1024 slots, which leaves room for
// more CTAs per SM. Every segment's hash has HSTRIDE slots in HBM.
template <int RULE>
struct HashCfg {
    static constexpr int BITS = RULE == RULE_MAXP ? 10 : 11;
    static constexpr int SLOTS = 1 << BITS;
    static constexpr int FILL = BITS == 11 ? 1400 : SLOTS * 11 / 16;
};
constexpr int HSTRIDE = 2048;

size_t seg_hash_bytes() { return (size_t)HSTRIDE * sizeof(unsigned long long); }

// ---- per-segment step log -------------------------------------------------------
// Every step of every speculative chain of a segment, in the order taken:
// record = (position | chain << 57, k << 32 | d): the chain visits position,
// position + d, ..., position + (k - 1) d, and goes on at position + k d.
// A chain's records appear in increasing position order. The output kernel
// replays the true chain from these records instead of stepping again.
// (A.logcap records per segment, set by the host)
// then the stitch walks: SWPW records per warp of the stitch kernel
constexpr int SWPW = 64;
constexpr int SWCAP = SWPW * (NL / 32);
size_t seg_log_bytes(uint32_t logcap) { return (size_t)(logcap + SWCAP) * 16; }

__device__ __forceinline__ void log_step(const ChainLaunch& A, uint64_t item, unsigned int* log_n, uint32_t chain,
                                         uint64_t pos, uint32_t k, uint64_t d) {
    const unsigned int i = atomicAdd(log_n, 1u);
    if (i < A.logcap) {
        ulonglong2 r;
        r.x = pos | ((unsigned long long)chain << 57);
        r.y = ((unsigned long long)k << 32) | (uint32_t)d;
        reinterpret_cast<ulonglong2*>(A.plog)[item * (uint64_t)(A.logcap + SWCAP) + i] = r;
    }
}

template <int RULE>
__device__ __forceinline__ uint32_t hslot(uint32_t key) {
    return (key * 2654435761u) >> (32 - HashCfg<RULE>::BITS);
}
constexpr uint32_t H_INSERTED = 0xFFFFFFFFu, H_FULL = 0xFFFFFFFEu;

// insert; returns H_INSERTED, H_FULL, or the value already stored for key
template <int RULE>
__device__ __forceinline__ uint32_t hinsert(unsigned long long* ht, unsigned int* fill, uint32_t key, uint32_t val) {
    if (*reinterpret_cast<volatile unsigned int*>(fill) >= (unsigned)HashCfg<RULE>::FILL) return H_FULL;
    const unsigned long long ent = ((unsigned long long)key << 32) | val;
    uint32_t s = hslot<RULE>(key);
    for (int i = 0; i < 64; i++) {
        unsigned long long prev = atomicCAS(&ht[s], 0ull, ent);
        if (prev == 0ull) {
            atomicAdd(fill, 1u);
            return H_INSERTED;
        }
        if ((uint32_t)(prev >> 32) == key) return (uint32_t)prev;
        s = (s + 1) & (HashCfg<RULE>::SLOTS - 1);
    }
    return H_FULL;
}

// value stored for key, or ~0u
template <int RULE>
__device__ __forceinline__ uint32_t hfind(const unsigned long long* ht, uint32_t key) {
    uint32_t s = hslot<RULE>(key);
    for (int i = 0; i < 64; i++) {
        const unsigned long long e = ht[s];
        if ((uint32_t)(e >> 32) == key) return (uint32_t)e;
        if (e == 0ull) return ~0u;
        s = (s + 1) & (HashCfg<RULE>::SLOTS - 1);
    }
    return ~0u;
}

__device__ __forceinline__ void stat_add(const ChainLaunch& A, int k, unsigned long long v) {
    if (A.stats && v) atomicAdd(&A.ctrl->stats[k], v);
}

// ---- bounded waits -------------------------------------------------------------

__device__ bool wait_flag_thread(const unsigned int* f, uint32_t epoch, const ChainLaunch& A, uint64_t item) {
    if (ld_acquire(f) == epoch) return true;
    uint64_t t0 = gtimer_ns();
    for (;;) {
        if (ld_acquire(f) == epoch) return true;
        if (ld_volatile(&A.ctrl->err)) return false;
        if (gtimer_ns() - t0 > A.timeout_ns) {
            atomicOr(&A.ctrl->err, ERR_TIMEOUT);
            A.ctrl->err_info = item;
            return false;
        }
        __nanosleep(100);
    }
}

// ---- k_spec: speculate and stitch ------------------------------------------------

constexpr int KS = 1;          // per-thread steps per round before the live chains are compacted

template <int RULE>
struct SpecShared {
    unsigned long long ht[HashCfg<RULE>::SLOTS];
    unsigned int fill;
    unsigned int log_n;            // records in the segment's step log
    unsigned int nq;               // live chains (compacted into threads [0, nq))
    unsigned int nq2;
    unsigned int q_lane[2][NL];    // chain id, position, count of the live chains
    unsigned long long q_s[2][NL];
    unsigned int q_c[2][NL];
    unsigned long long X[NL];
    unsigned int cnt[NL];
    int mg[NL];            // chain this one merged into, or -1
    unsigned int mc[NL];   // its own count at the merge position
    unsigned int mi[NL];   // index of that position in the target chain
    unsigned long long geo[5];
    unsigned long long item;
    int ok;
};

template <int RULE>
__global__ void __launch_bounds__(NL) k_spec(ChainLaunch A) {
    extern __shared__ __align__(16) uint8_t dsm[];  // staged summaries: m[win], a[win]
    __shared__ SpecShared<RULE> sh;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t epoch = ld_volatile(&A.ctrl->epoch);
    const uint64_t n_items = A.n_items_dev ? *reinterpret_cast<const volatile unsigned long long*>(A.n_items_dev)
                                           : A.n_items;
    const Prm P{A.w, A.mn, A.mx};
    const RawView R{A.base, A.inv};
    for (;;) {
        long long t_mark = clock64();
        if (tid == 0) {
            sh.item = atomicAdd(&A.ctrl->ticket, 1ull);
            sh.ok = ld_volatile(&A.ctrl->err) == 0;
        }
        for (int i = tid; i < HashCfg<RULE>::SLOTS; i += NL) sh.ht[i] = 0ull;
        if (tid == 0) {
            sh.fill = 0;
            sh.log_n = 0;
        }
        __syncthreads();
        const uint64_t item = sh.item;
        if (item >= n_items || !sh.ok) break;
        if (tid < 64) {  // warp 0: seg_lo, warp 1: seg_hi
            const Geo g = seg_geo(A, item, lane, tid >> 5);
            if (tid == 0) {
                sh.geo[0] = g.seg_lo; sh.geo[2] = g.flo; sh.geo[3] = g.fhi;
                sh.geo[4] = g.first ? GEO_FIRST : 0u;
            }
            if (tid == 32) sh.geo[1] = g.seg_hi;
        }
        __syncthreads();
        if (tid == 0) {  // empty: the bounds met (a quiet run pushed both); last: it ends the file
            if (sh.geo[1] < sh.geo[0]) sh.geo[1] = sh.geo[0];
            const bool empty = sh.geo[1] == sh.geo[0];
            sh.geo[4] |= (empty ? GEO_EMPTY : 0u) | (!empty && sh.geo[1] == sh.geo[3] ? GEO_LAST : 0u);
        }
        __syncthreads();
        const uint64_t seg_lo = sh.geo[0], seg_hi = sh.geo[1], flo = sh.geo[2], fhi = sh.geo[3];
        const uint32_t geo = (uint32_t)sh.geo[4];
        const bool first = geo & GEO_FIRST, last = geo & GEO_LAST, empty = geo & GEO_EMPTY;
        SegState* me = &A.st[item];
        const bool hold = (int64_t)item == A.hold_item;

        // stage block summaries of [seg_lo, seg_lo + win * 64)
        SumView S{A.smax, A.sarg, dsm, dsm + A.win, 0, 0, A.ssup};
        if (RULE == RULE_RAM || RULE == RULE_AE || RULE == RULE_MAXP) {
            uint64_t wb0 = (seg_lo >> 6) & ~15ull;
            uint64_t wn = A.win;
            if (wb0 + wn > A.nblk_pad) wn = A.nblk_pad > wb0 ? ((A.nblk_pad - wb0) & ~15ull) : 0;
            for (uint64_t o = (uint64_t)tid * 16; o < wn; o += NL * 16) {
                *reinterpret_cast<uint4*>(dsm + o) = *reinterpret_cast<const uint4*>(A.smax + wb0 + o);
                if (RULE != RULE_MAXP)
                    *reinterpret_cast<uint4*>(dsm + A.win + o) = *reinterpret_cast<const uint4*>(A.sarg + wb0 + o);
            }
            S.wb0 = wb0;
            S.wn = wn;
        }
        const Win W{dsm, dsm + A.win, S.wb0 << 6, (uint32_t)(S.wn << 6)};
        __syncthreads();

        auto lap = [&](int k) {
            if (A.stats && tid == 0) {
                const long long t = clock64();
                stat_add(A, k, (unsigned long long)(t - t_mark));
                t_mark = t;
            }
        };
        lap(STAT_CYC_SETUP);
        // ---- speculative chains
        uint64_t x = ~0ull;
        uint32_t c = 0;
        int mg = -1;
        uint32_t mi = 0;
        long long t_surv0 = 0;
        if (empty) {
            // nothing inside: the nearest non-empty predecessor's exits pass
            // through unchanged (copied by the stitch kernel)
        } else {
            uint64_t start = ~0ull;
            if (first) {
                if (tid == 0) start = flo;
            } else {
                // threads beyond `starts` repeat a start: they merge on their first hash insert
                const uint32_t ns = A.starts;
                uint64_t d = umin64(A.span, seg_hi - seg_lo) / ns;
                start = seg_lo + (uint64_t)((uint32_t)tid % ns) * (d ? d : 1);
            }
            // rounds of KS per-thread steps; live chains are compacted into the
            // lowest threads after every round so that idle warps issue nothing
            uint32_t tsteps = 0;
            if (tid == 0) sh.nq = 0;
            __syncthreads();
            if (start < seg_hi) {
                const unsigned q = atomicAdd(&sh.nq, 1u);
                sh.q_lane[0][q] = (unsigned)tid;
                sh.q_s[0][q] = start;
                sh.q_c[0][q] = 0;
            }
            sh.mg[tid] = -1;
            sh.X[tid] = ~0ull;
            sh.cnt[tid] = 0;
            __syncthreads();
            int buf = 0;
            const bool rec = !first;
            const long long t_r0 = clock64();
            uint32_t rounds = 0;
            for (;;) {
                const unsigned nq = sh.nq;
                if (nq <= A.warp_chains) break;  // the rest: one warp per chain
                rounds++;
                if (tid == 0) sh.nq2 = 0;
                __syncthreads();
                if ((unsigned)tid < nq) {
                    const unsigned l = sh.q_lane[buf][tid];
                    uint64_t s = sh.q_s[buf][tid];
                    uint32_t c = sh.q_c[buf][tid];
                    bool alive = true, recl = rec;
                    for (int r = 0; r < KS; r++) {
                        if (recl) {
                            const uint32_t hr = c < 0xFFFFu ? hinsert<RULE>(sh.ht, &sh.fill, (uint32_t)(s - seg_lo) + 1u,
                                                                       (l << 16) | c)
                                                            : H_FULL;
                            if (hr == H_FULL) {
                                recl = false;
                            } else if (hr != H_INSERTED) {  // another chain was here first: same chain from now on
                                sh.mg[l] = (int)(hr >> 16);
                                sh.mc[l] = c;
                                sh.mi[l] = hr & 0xFFFFu;
                                alive = false;
                                stat_add(A, STAT_MERGES, 1);
                                break;
                            }
                        }
                        uint32_t k;
                        uint64_t dd;
                        const uint64_t s0 = s;
                        s = advance<RULE>(S, R, P, flo - A.wctx, fhi, s, seg_hi, &k, &dd);
                        log_step(A, item, &sh.log_n, l, s0, k, dd);
                        c += k;
                        tsteps++;
                        if (s >= seg_hi) {
                            sh.X[l] = s;
                            sh.cnt[l] = c;
                            alive = false;
                            break;
                        }
                    }
                    if (alive) {
                        const unsigned q = atomicAdd(&sh.nq2, 1u);
                        sh.q_lane[buf ^ 1][q] = l;
                        sh.q_s[buf ^ 1][q] = s;
                        sh.q_c[buf ^ 1][q] = c;
                    }
                }
                __syncthreads();
                if (tid == 0) sh.nq = sh.nq2;
                buf ^= 1;
                __syncthreads();
            }
            const long long t_r1 = clock64();
            t_surv0 = t_r1;
            if (A.stats && tid == 0) {
                stat_add(A, STAT_ROUNDS, rounds);
                stat_add(A, STAT_CYC_ROUNDS, (unsigned long long)(t_r1 - t_r0));
            }
            if (A.stats) {
                unsigned long long tot = tsteps;
                for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(FULL, tot, o);
                if (lane == 0) stat_add(A, STAT_THREAD_STEPS, tot);
                if (tid == 0) {
                    stat_add(A, STAT_SEGMENTS, 1);
                    stat_add(A, STAT_SURVIVORS, sh.nq);
                    if (sh.fill >= (unsigned)HashCfg<RULE>::FILL) stat_add(A, STAT_HASH_FULL, 1);
                }
            }
            // the last chains, one warp each (every step shared by the 32 lanes);
            // a warp that finishes a chain takes the next one
            if (tid == 0) sh.nq2 = NW;
            __syncthreads();
            for (unsigned q = (unsigned)(tid >> 5); q < sh.nq;) {
                const unsigned l = sh.q_lane[buf][q];
                uint64_t v = sh.q_s[buf][q];
                uint32_t cc = sh.q_c[buf][q];
                bool recq = rec;
                int qmg = -1;
                uint32_t qmi = 0;
                while (v < seg_hi) {
                    if (recq) {
                        uint32_t hr = H_FULL;
                        if (lane == 0 && cc < 0xFFFFu)
                            hr = hinsert<RULE>(sh.ht, &sh.fill, (uint32_t)(v - seg_lo) + 1u, (l << 16) | cc);
                        hr = __shfl_sync(FULL, hr, 0);
                        if (hr == H_FULL) {
                            recq = false;
                        } else if (hr != H_INSERTED) {
                            qmg = (int)(hr >> 16);
                            qmi = hr & 0xFFFFu;
                            break;
                        }
                    }
                    uint32_t k;
                    uint64_t dd;
                    const uint64_t v0 = v;
                    v = f_advance<RULE>(W, S, R, P, flo - A.wctx, fhi, v, seg_hi, &k, &dd);
                    if (lane == 0) log_step(A, item, &sh.log_n, l, v0, k, dd);
                    cc += k;
                    if (lane == 0) stat_add(A, STAT_WARP_STEPS, 1);
                }
                if (lane == 0) {
                    sh.mg[l] = qmg;
                    sh.mc[l] = cc;
                    sh.mi[l] = qmi;
                    if (qmg < 0) {
                        sh.X[l] = v;
                        sh.cnt[l] = cc;
                    }
                    q = atomicAdd(&sh.nq2, 1u);
                }
                q = __shfl_sync(FULL, q, 0);
            }
        }
        if (empty) {
            sh.mg[tid] = -1;
            sh.X[tid] = x;
            sh.cnt[tid] = 0;
            if (tid == 0) stat_add(A, STAT_EMPTY, 1);
        }
        __syncthreads();
        if (A.stats && tid == 0 && !empty) stat_add(A, STAT_CYC_SURV, (unsigned long long)(clock64() - t_surv0));
        lap(STAT_CYC_THREADS);
        __syncthreads();
        mg = sh.mg[tid];
        x = sh.X[tid];
        c = sh.cnt[tid];
        if (mg >= 0) {  // follow the merges to a chain that ran to the end
            uint32_t acc = 0;
            int l = tid;
            while (sh.mg[l] >= 0) {
                acc += sh.mc[l] - sh.mi[l];
                l = sh.mg[l];
            }
            x = sh.X[l];
            c = acc + sh.cnt[l];
        }
        __syncthreads();
        me->X[tid] = x;
        me->cnt[tid] = c;
        if (tid == 0) {
            me->seg_lo = seg_lo; me->seg_hi = seg_hi; me->flo = flo; me->fhi = fhi; me->geo = geo;
            me->log_n = sh.log_n;
        }
        // the position hash goes to HBM for the stitch kernels
        if (!first && !empty) {
            uint4* dst = reinterpret_cast<uint4*>(A.hash + item * (uint64_t)HSTRIDE);
            const uint4* src = reinterpret_cast<const uint4*>(sh.ht);
            for (int i = tid; i < HashCfg<RULE>::SLOTS / 2; i += NL) dst[i] = src[i];
        }
        __syncthreads();
        if (!sh.ok) break;
        if (tid == 0) {
            __threadfence();
            if (!hold) st_release(&me->flagA, epoch);
        }
        lap(STAT_CYC_WARPS);
    }
}

// ---- stitching (after every segment has speculated: no waits) --------------------

// Nearest non-empty segment before `item` in its file (empty segments pass
// positions and chains through unchanged). item is not the first of its file.
__device__ __forceinline__ uint64_t nonempty_pred(const ChainLaunch& A, uint64_t item) {
    uint64_t q = item - 1;
    while (q > 0 && (A.st[q].geo & GEO_EMPTY) && !(A.st[q].geo & GEO_FIRST)) q--;
    return q;
}

// Follow the chain from e (every lane of the warp computes the same steps)
// until it lands on a hashed position of a chain of this segment, or reaches
// seg_hi. Returns the table encoding; *ux receives the exit when no chain was
// met (0 otherwise). ht, X, cnt: this segment's hash, exits and counts.
template <int RULE>
__device__ uint32_t stitch_walk(const ChainLaunch& A, const SumView& S, const RawView& R, const Prm& P,
                                const unsigned long long* ht, const unsigned long long* X, const unsigned int* cnt,
                                uint64_t seg_lo, uint64_t seg_hi, uint64_t wflo, uint64_t fhi, bool last, uint64_t e,
                                uint64_t* ux, uint64_t item, ulonglong2* slog = nullptr, uint32_t* slog_n = nullptr,
                                uint32_t slog_cap = 0) {
    const int lane = threadIdx.x & 31;
    uint32_t nsteps = 0;
    uint64_t v = e;
    uint32_t ne = 0, res = STAB_UNKNOWN;
    while (v < seg_hi) {
        const uint32_t hv = hfind<RULE>(ht, (uint32_t)(v - seg_lo) + 1u);
        if (hv != ~0u) {
            const uint32_t m = hv >> 16, idx = hv & 0xFFFFu;
            res = stab_enc(m, ne + cnt[m] - idx + (last ? 1u : 0u));
            break;
        }
        uint32_t k;
        uint64_t dd;
        const uint64_t v0 = v;
        v = w_advance<RULE>(S, R, P, wflo, fhi, v, seg_hi, &k, &dd);
        // the step goes to the walk's log (same record format as the speculation log)
        if (slog) {
            if (lane == 0 && *slog_n < slog_cap)
                slog[*slog_n] = make_ulonglong2(v0, ((unsigned long long)k << 32) | (uint32_t)dd);
            (*slog_n)++;
        }
        ne += k;
        nsteps++;
        if (lane == 0) stat_add(A, STAT_STITCH_STEPS, 1);
    }
    *ux = 0;
    if (res == STAB_UNKNOWN) {
        // ended at or past seg_hi: does it end on one of the chains' exits?
        uint32_t found = NL;
#pragma unroll
        for (int j = 0; j < NL / 32; j++) {
            const uint32_t b = __ballot_sync(FULL, X[j * 32 + lane] == v);
            if (b && found == NL) found = (uint32_t)(j * 32 + __ffs((int)b) - 1);
        }
        res = found < NL ? stab_enc(found, ne + (last ? 1u : 0u))
                         : (STAB_UNKNOWN | ((ne + (last ? 1u : 0u)) & 0x7FFFFFu));
        *ux = v;
    }
    if (lane == 0) {
        stat_add(A, STAT_STITCH_WALKS, 1);
        if (res & STAB_UNKNOWN) stat_add(A, STAT_UNKNOWN, 1);
        if (A.stats && nsteps > 64) {
            stat_add(A, STAT_STITCH_LONG, 1);
            atomicMax(&A.ctrl->stats[STAT_STITCH_MAXW], ((unsigned long long)nsteps << 32) | (item & 0xFFFFFFFFull));
        }
    }
    return res;
}

template <int RULE>
struct StitchShared {
    unsigned long long ht[HashCfg<RULE>::SLOTS];
    unsigned long long X[NL];
    unsigned int cnt[NL];
    int ok;
};

// Load a segment's hash, exits and counts into shared memory.
template <int RULE>
__device__ __forceinline__ void load_segment(const ChainLaunch& A, uint64_t item, StitchShared<RULE>& sh) {
    const int tid = threadIdx.x;
    const uint4* src = reinterpret_cast<const uint4*>(A.hash + item * (uint64_t)HSTRIDE);
    uint4* dst = reinterpret_cast<uint4*>(sh.ht);
    constexpr int PER = HashCfg<RULE>::SLOTS / 2 / NL;  // 16-byte loads per thread, all in flight at once
    static_assert(HashCfg<RULE>::SLOTS / 2 % NL == 0, "hash rows split evenly over the threads");
    uint4 r[PER];
#pragma unroll
    for (int k = 0; k < PER; k++) r[k] = src[tid + k * NL];
    const unsigned long long x = A.st[item].X[tid];
    const unsigned int c = A.st[item].cnt[tid];
#pragma unroll
    for (int k = 0; k < PER; k++) dst[tid + k * NL] = r[k];
    sh.X[tid] = x;
    sh.cnt[tid] = c;
}

// k_stitch: table "predecessor chain -> (chain, boundaries in this segment)"
// for every segment; empty segments take their predecessor's exits.
template <int RULE>
__global__ void __launch_bounds__(NL) k_stitch(ChainLaunch A) {
    __shared__ StitchShared<RULE> sh;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t epoch = ld_volatile(&A.ctrl->epoch);
    const uint64_t n_items = A.n_items_dev ? *reinterpret_cast<const volatile unsigned long long*>(A.n_items_dev)
                                           : A.n_items;
    const Prm P{A.w, A.mn, A.mx};
    const RawView R{A.base, A.inv};
    const SumView S{A.smax, A.sarg, nullptr, nullptr, 0, 0, A.ssup};
    for (uint64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const long long t0 = clock64();
        if (tid == 0) {
            sh.ok = ld_volatile(&A.ctrl->err) == 0;
            // every segment published its state before this kernel started,
            // unless a test holds one back: then this bounded wait runs out
            if (sh.ok && !wait_flag_thread(&A.st[item].flagA, epoch, A, item)) sh.ok = 0;
        }
        __syncthreads();
        if (!sh.ok) break;
        SegState* me = &A.st[item];
        const uint32_t geo = me->geo;
        const bool first = geo & GEO_FIRST, last = geo & GEO_LAST, empty = geo & GEO_EMPTY;
        uint32_t tab;
        unsigned long long unk = ~0ull;  // no position: slots of chains that never ran stay so
        unsigned short swf = 0, swc = 0xFFFFu;  // this slot's logged walk
        if (first) {
            tab = stab_enc(0, me->cnt[0] - 1 + (last ? 1u : 0u)) | STAB_CONST;
        } else if (empty) {
            tab = stab_enc((uint32_t)tid, 0);
            me->X[tid] = A.st[nonempty_pred(A, item)].X[tid];
        } else {
            const uint64_t p = nonempty_pred(A, item);
            const uint64_t xp = A.st[p].X[tid];
            load_segment(A, item, sh);
            __syncthreads();
            const uint64_t seg_lo = me->seg_lo, seg_hi = me->seg_hi, flo = me->flo, fhi = me->fhi;
            tab = STAB_UNKNOWN;
            uint32_t todo = __ballot_sync(FULL, xp != ~0ull);
            // this warp's walks go to its part of the segment's stitch log
            ulonglong2* slog = reinterpret_cast<ulonglong2*>(A.plog) + item * (uint64_t)(A.logcap + SWCAP) + A.logcap +
                               (uint64_t)(tid >> 5) * SWPW;
            uint32_t slog_n = 0;
            while (todo) {
                const int ld = __ffs((int)todo) - 1;
                const uint64_t e = __shfl_sync(FULL, xp, ld);
                const uint32_t same = __ballot_sync(FULL, xp == e) & todo;
                uint64_t ux;
                const uint32_t first_rec = slog_n;
                const uint32_t res = stitch_walk<RULE>(A, S, R, P, sh.ht, sh.X, sh.cnt, seg_lo, seg_hi, flo - A.wctx, fhi,
                                                       last, e, &ux, item, slog, &slog_n, SWPW);
                if ((same >> lane) & 1u) {
                    tab = res;
                    unk = ux;
                    swf = (unsigned short)((tid >> 5) * SWPW + first_rec);
                    swc = slog_n <= (uint32_t)SWPW ? (unsigned short)(slog_n - first_rec) : (unsigned short)0xFFFFu;
                }
                todo &= ~same;
            }
        }
        me->table[tid] = tab;
        me->unk_exit[tid] = unk;
        me->sw_first[tid] = swf;
        me->sw_cnt[tid] = swc;
        __syncthreads();
        if (A.stats && tid == 0) stat_add(A, STAT_CYC_STITCH, (unsigned long long)(clock64() - t0));
    }
}

// k_ures: positions that reach a segment off every chain (its nearest
// non-empty predecessor's uncovered exits) are followed here, so that the
// resolution kernels need not walk whole segments.
template <int RULE>
__global__ void __launch_bounds__(NL) k_ures(ChainLaunch A) {
    __shared__ StitchShared<RULE> sh;
    __shared__ int any;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint64_t n_items = A.n_items_dev ? *reinterpret_cast<const volatile unsigned long long*>(A.n_items_dev)
                                           : A.n_items;
    if (ld_volatile(&A.ctrl->err)) return;
    const Prm P{A.w, A.mn, A.mx};
    const RawView R{A.base, A.inv};
    const SumView S{A.smax, A.sarg, nullptr, nullptr, 0, 0, A.ssup};
    for (uint64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        SegState* me = &A.st[item];
        const uint32_t geo = me->geo;
        const bool first = geo & GEO_FIRST, last = geo & GEO_LAST, empty = geo & GEO_EMPTY;
        if (first || empty) {
            if (tid == 0) me->ures_n = 0;
            continue;
        }
        const SegState* qs = &A.st[nonempty_pred(A, item)];
        const uint32_t t = qs->table[tid];
        const bool u = (t & STAB_UNKNOWN) && !(t & STAB_CONST) && qs->unk_exit[tid] != ~0ull;
        if (tid == 0) any = 0;
        __syncthreads();
        if (u) any = 1;
        __syncthreads();
        if (!any) {
            if (tid == 0) me->ures_n = 0;
            __syncthreads();
            continue;
        }
        load_segment(A, item, sh);
        __syncthreads();
        if (tid < 32) {
            const uint64_t seg_lo = me->seg_lo, seg_hi = me->seg_hi, flo = me->flo, fhi = me->fhi;
            uint64_t up[NL / 32];
#pragma unroll
            for (int j = 0; j < NL / 32; j++) {
                const uint32_t tj = qs->table[lane + 32 * j];
                // ~0: the predecessor's chain in this slot never ran (nothing to follow)
                up[j] = ((tj & STAB_UNKNOWN) && !(tj & STAB_CONST)) ? qs->unk_exit[lane + 32 * j] : ~0ull;
            }
            uint32_t nu = 0;
            for (int j = 0; j < NL / 32; j++) {
                uint32_t todo = __ballot_sync(FULL, up[j] != ~0ull);
                while (todo && nu < (uint32_t)NU) {
                    const int ld = __ffs((int)todo) - 1;
                    const uint64_t e = __shfl_sync(FULL, up[j], ld);
#pragma unroll
                    for (int jj = 0; jj < NL / 32; jj++)
                        if (up[jj] == e) up[jj] = ~0ull;
                    todo = __ballot_sync(FULL, up[j] != ~0ull);
                    uint64_t ux;
                    const uint32_t res = stitch_walk<RULE>(A, S, R, P, sh.ht, sh.X, sh.cnt, seg_lo, seg_hi, flo - A.wctx, fhi,
                                                           last, e, &ux, item);
                    if (lane == 0) {
                        me->ures_pos[nu] = e;
                        me->ures_exit[nu] = ux;
                        me->ures_val[nu] = res;
                    }
                    nu++;
                }
            }
            if (lane == 0) me->ures_n = nu;
        }
        __syncthreads();
    }
}

// ---- following the true chain through one segment (global summaries) ----------

// Walk the chain from position v through segment st (warp-uniform). Returns
// the number of boundaries inside and the exit; *slot receives the chain of
// the segment that ends on the same exit, or NONE.
template <int RULE>
__device__ uint32_t follow(const ChainLaunch& A, const SegState* st, uint64_t v, uint64_t* exit, uint32_t* slot) {
    const SumView S{A.smax, A.sarg, nullptr, nullptr, 0, 0, A.ssup};
    const RawView R{A.base, A.inv};
    const Prm P{A.w, A.mn, A.mx};
    const uint64_t seg_hi = st->seg_hi, wflo = st->flo - A.wctx, fhi = st->fhi;
    const bool last = st->geo & GEO_LAST;
    uint32_t n = 0;
    while (v < seg_hi) {
        uint32_t k;
        uint64_t dd;
        v = w_advance<RULE>(S, R, P, wflo, fhi, v, seg_hi, &k, &dd);
        n += k;
    }
    if (last) n++;
    *exit = v;
    const int lane = threadIdx.x & 31;
    uint32_t found = NONE;
#pragma unroll
    for (int j = 0; j < NL / 32; j++) {
        uint32_t b = __ballot_sync(FULL, st->X[j * 32 + lane] == v);
        if (b && found == NONE) found = (uint32_t)(j * 32 + __ffs((int)b) - 1);
    }
    *slot = found;
    return n;
}

// Table entry for a state entering segment st: `slot` is the chain of the
// previous segment (or NONE: then only the position is known).
__device__ __forceinline__ uint32_t lookup(uint32_t t0, const uint32_t t[NL / 32], uint32_t slot) {
    if (__shfl_sync(FULL, t0, 0) & STAB_CONST) return __shfl_sync(FULL, t0, 0);
    const uint32_t s = slot < NL ? slot : 0;
    uint32_t v = 0;
#pragma unroll
    for (int j = 0; j < NL / 32; j++) {
        uint32_t x = __shfl_sync(FULL, t[j], (int)(s & 31));
        if ((s >> 5) == (uint32_t)j) v = x;
    }
    return slot < NL ? v : (STAB_UNKNOWN | 0x7FFFFFu);
}

// One step of the true state through segment i, given its table entry e for
// the state and its geometry word geo. (slot, pos): chain of the previous
// segment, or NONE and the exact position. Returns the boundaries inside
// segment i.
template <int RULE>
__device__ uint32_t step_with(const ChainLaunch& A, uint64_t i, uint32_t e, uint32_t geo, uint32_t* slot,
                              uint64_t* pos) {
    const SegState* st = &A.st[i];
    if (geo & GEO_EMPTY) return 0;  // nothing inside: the state passes through
    if (!(e & STAB_UNKNOWN) || (e & STAB_CONST)) {
        *slot = stab_slot(e);
        *pos = 0;
        return stab_count(e);
    }
    if (*slot < NL) {  // the stitch followed this entry to the end without meeting a chain
        *pos = st->unk_exit[*slot];
        *slot = NONE;
        return stab_count(e);
    }
    // off every chain at *pos: the segment may have followed that position already
    const int lane = threadIdx.x & 31;
    const uint32_t nu = st->ures_n;
    const uint32_t hit = __ballot_sync(FULL, (uint32_t)lane < nu && lane < NU && st->ures_pos[lane < NU ? lane : 0] == *pos);
    if (hit) {
        const int l = __ffs((int)hit) - 1;
        const uint32_t v = st->ures_val[l];
        if (!(v & STAB_UNKNOWN)) {
            *slot = stab_slot(v);
            *pos = 0;
        } else {
            *slot = NONE;
            *pos = st->ures_exit[l];
        }
        return stab_count(v);
    }
    uint64_t ex;
    uint32_t sl;
    uint32_t n = follow<RULE>(A, st, *pos, &ex, &sl);
    if (lane == 0) stat_add(A, STAT_SCAN_FOLLOWS, 1);
    *slot = sl;
    *pos = ex;
    return n;
}

// ---- k_compose: group composites ---------------------------------------------------

template <int RULE>
__global__ void __launch_bounds__(32) k_compose(ChainLaunch A) {
    if (ld_volatile(&A.ctrl->err)) return;  // a speculation wait ran out: nothing to resolve
    static_assert(NL == 128, "composition below assumes 4 table entries per lane");
    const int lane = threadIdx.x;
    const uint64_t n_items = A.n_items_dev ? *reinterpret_cast<const volatile unsigned long long*>(A.n_items_dev)
                                           : A.n_items;
    const uint64_t ngroups = (n_items + A.gs - 1) / A.gs;
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const uint64_t i0 = g * A.gs, i1 = umin64(i0 + A.gs, n_items);
        uint32_t sl[4];
        unsigned long long cn[4], ps[4];  // ps: position while sl == NONE (off every chain)
#pragma unroll
        for (int j = 0; j < 4; j++) { sl[j] = (uint32_t)(lane + 32 * j); cn[j] = 0; ps[j] = 0; }
        // tables of the next PD segments in flight (slot d holds segment i with (i - i0) % PD == d)
        constexpr uint64_t PD = 8;
        uint32_t nt[PD][4], ngeo[PD];
#pragma unroll
        for (uint64_t d = 0; d < PD; d++)
            if (i0 + d < i1) {
#pragma unroll
                for (int j = 0; j < 4; j++) nt[d][j] = A.st[i0 + d].table[lane + 32 * j];
                ngeo[d] = A.st[i0 + d].geo;
            }
        for (uint64_t ib = i0; ib < i1; ib += PD)
#pragma unroll
        for (uint64_t d = 0; d < PD; d++) {
            const uint64_t i = ib + d;
            if (i >= i1) break;
            uint32_t t[4];
#pragma unroll
            for (int j = 0; j < 4; j++) t[j] = nt[d][j];
            const uint32_t geo = ngeo[d];
            if (i + PD < i1) {  // prefetch the table PD segments ahead
#pragma unroll
                for (int j = 0; j < 4; j++) nt[d][j] = A.st[i + PD].table[lane + 32 * j];
                ngeo[d] = A.st[i + PD].geo;
            }
            if (geo & GEO_EMPTY) continue;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t e = lookup(t[0], t, sl[j]);
                if (sl[j] == UNRESOLVED) continue;
                if (!(e & STAB_UNKNOWN) || (e & STAB_CONST)) {
                    sl[j] = stab_slot(e);
                    cn[j] += stab_count(e);
                } else if (sl[j] < NL) {  // the stitch met no chain: continue from its exit
                    ps[j] = A.st[i].unk_exit[sl[j]];
                    cn[j] += stab_count(e);
                    sl[j] = NONE;
                } else {  // entering off every chain: did the segment follow this position?
                    const SegState* st = &A.st[i];
                    const uint32_t nu = umin64(st->ures_n, NU);
                    uint32_t v = STAB_UNKNOWN, f = 0;
                    for (uint32_t u = 0; u < nu; u++)
                        if (st->ures_pos[u] == ps[j]) { v = st->ures_val[u]; f = 1; ps[j] = st->ures_exit[u]; break; }
                    if (!f) {
                        sl[j] = UNRESOLVED;
                    } else if (!(v & STAB_UNKNOWN)) {
                        sl[j] = stab_slot(v);
                        cn[j] += stab_count(v);
                    } else {
                        cn[j] += stab_count(v);  // still off every chain, at the new exit
                    }
                }
            }
        }
        GroupState* gs = reinterpret_cast<GroupState*>(A.groups) + g;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            gs->slot[lane + 32 * j] = sl[j] == NONE ? UNRESOLVED : sl[j];
            gs->count[lane + 32 * j] = cn[j];
        }
    }
}

// ---- k_scan: the true state entering every group -------------------------------------

template <int RULE>
__global__ void __launch_bounds__(32) k_scan(ChainLaunch A) {
    if (ld_volatile(&A.ctrl->err)) return;  // a speculation wait ran out: nothing to resolve
    const int lane = threadIdx.x;
    const uint64_t n_items = A.n_items_dev ? *reinterpret_cast<const volatile unsigned long long*>(A.n_items_dev)
                                           : A.n_items;
    const uint64_t ngroups = (n_items + A.gs - 1) / A.gs;
    GroupState* G = reinterpret_cast<GroupState*>(A.groups);
    uint32_t slot = NONE;
    uint64_t pos = A.lo, incl = 0;
    constexpr int B = 4;  // composites prefetched per round
    for (uint64_t g0 = 0; g0 < ngroups; g0 += B) {
        uint32_t gsl[B][4], gfirst[B];
        unsigned long long gcn[B][4];
#pragma unroll
        for (int b = 0; b < B; b++) {
            const uint64_t g = g0 + b;
            if (g < ngroups) {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    gsl[b][j] = G[g].slot[lane + 32 * j];
                    gcn[b][j] = G[g].count[lane + 32 * j];
                }
                gfirst[b] = A.st[g * A.gs].geo & GEO_FIRST;
            }
        }
#pragma unroll
        for (int b = 0; b < B; b++) {
            const uint64_t g = g0 + b;
            if (g >= ngroups) break;
            if (lane == 0) {
                G[g].entry_slot = slot;
                G[g].entry_pos = slot < NL ? 0 : pos;
                G[g].entry_incl = incl;
            }
            const uint32_t s = gfirst[b] ? 0u : slot;
            uint32_t ns = UNRESOLVED;
            unsigned long long nc = 0;
            if (s < NL) {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    uint32_t a = __shfl_sync(FULL, gsl[b][j], (int)(s & 31));
                    unsigned long long c = __shfl_sync(FULL, gcn[b][j], (int)(s & 31));
                    if ((s >> 5) == (uint32_t)j) { ns = a; nc = c; }
                }
            }
            if (ns != UNRESOLVED) {
                slot = ns;
                incl += nc;
            } else {
                // follow the group segment by segment (tables prefetched one ahead)
                const uint64_t i0 = g * A.gs, i1 = umin64(i0 + A.gs, n_items);
                uint32_t nt[4], ng = A.st[i0].geo;
#pragma unroll
                for (int j = 0; j < 4; j++) nt[j] = A.st[i0].table[lane + 32 * j];
                for (uint64_t i = i0; i < i1; i++) {
                    uint32_t t[4];
                    const uint32_t geo = ng;
#pragma unroll
                    for (int j = 0; j < 4; j++) t[j] = nt[j];
                    if (i + 1 < i1) {
#pragma unroll
                        for (int j = 0; j < 4; j++) nt[j] = A.st[i + 1].table[lane + 32 * j];
                        ng = A.st[i + 1].geo;
                    }
                    const uint32_t e = lookup(t[0], t, slot);
                    incl += step_with<RULE>(A, i, e, geo, &slot, &pos);
                }
            }
        }
    }
    if (lane == 0) {
        A.ctrl->total = incl;
        if (A.d_count) *A.d_count = incl;
    }
}

// ---- k_settle: each segment's true entry and global offset -----------------------------

template <int RULE>
__global__ void __launch_bounds__(32) k_settle(ChainLaunch A) {
    if (ld_volatile(&A.ctrl->err)) return;  // a speculation wait ran out: nothing to resolve
    const int lane = threadIdx.x;
    const uint64_t n_items = A.n_items_dev ? *reinterpret_cast<const volatile unsigned long long*>(A.n_items_dev)
                                           : A.n_items;
    const uint64_t ngroups = (n_items + A.gs - 1) / A.gs;
    const GroupState* G = reinterpret_cast<const GroupState*>(A.groups);
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        uint32_t slot = G[g].entry_slot;
        uint64_t pos = G[g].entry_pos, incl = G[g].entry_incl;
        const uint64_t i0 = g * A.gs, i1 = umin64(i0 + A.gs, n_items);
        for (uint64_t b0 = i0; b0 < i1; b0 += 32) {
            // lane t records segment b0 + t: the state before it, its offset and count
            uint32_t my_slot = NONE, my_cnt = 0;
            uint64_t my_pos = 0, my_excl = 0;
            const uint32_t nb = (uint32_t)umin64(32, i1 - b0);
            // tables and geometry words of the next PD segments in flight (slot d
            // holds segment k with k % PD == d)
            constexpr uint32_t PD = 4;
            uint32_t nt[PD][4], ngeo[PD];
#pragma unroll
            for (uint32_t d = 0; d < PD; d++)
                if (d < nb) {
#pragma unroll
                    for (int j = 0; j < 4; j++) nt[d][j] = A.st[b0 + d].table[lane + 32 * j];
                    ngeo[d] = A.st[b0 + d].geo;
                }
            for (uint32_t k0 = 0; k0 < nb; k0 += PD) {
#pragma unroll
                for (uint32_t d = 0; d < PD; d++) {
                    const uint32_t k = k0 + d;
                    if (k < nb) {
                        const uint64_t i = b0 + k;
                        uint32_t t[4];
#pragma unroll
                        for (int j = 0; j < 4; j++) t[j] = nt[d][j];
                        const uint32_t geo = ngeo[d];
                        if (k + PD < nb) {
#pragma unroll
                            for (int j = 0; j < 4; j++) nt[d][j] = A.st[i + PD].table[lane + 32 * j];
                            ngeo[d] = A.st[i + PD].geo;
                        }
                        if (lane == (int)k) { my_slot = slot; my_pos = pos; my_excl = incl; }
                        const uint32_t e = lookup(t[0], t, slot);
                        const uint32_t n = step_with<RULE>(A, i, e, geo, &slot, &pos);
                        incl += n;
                        if (lane == (int)k) my_cnt = n;
                    }
                }
            }
            if ((uint32_t)lane < nb) {
                const uint64_t i = b0 + lane;
                SegState* st = &A.st[i];
                const uint32_t geo = st->geo;
                uint64_t entry = st->flo;
                if (!(geo & GEO_FIRST)) entry = my_slot < NL ? A.st[i - 1].X[my_slot] : my_pos;
                st->entry_pos = entry;
                st->entry_slot = !(geo & GEO_FIRST) && my_slot < NL ? my_slot : NONE;
                st->excl = my_excl;
                st->count = my_cnt;
            }
            __syncwarp();
        }
    }
}

// ---- k_output: write the true chain's boundaries -------------------------------------

template <int RULE>
__global__ void __launch_bounds__(32) k_output(ChainLaunch A) {
    if (ld_volatile(&A.ctrl->err)) return;  // a speculation wait ran out: nothing to resolve
    const int lane = threadIdx.x;
    const uint64_t n_items = A.n_items_dev ? *reinterpret_cast<const volatile unsigned long long*>(A.n_items_dev)
                                           : A.n_items;
    const Prm P{A.w, A.mn, A.mx};
    const RawView R{A.base, A.inv};
    for (uint64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const SegState* st = &A.st[item];
        const uint32_t geo = st->geo;
        const uint64_t seg_lo = st->seg_lo, seg_hi = st->seg_hi, flo = st->flo, fhi = st->fhi;
        const uint64_t excl = st->excl;
        const uint32_t cnt = st->count;
        const bool first = geo & GEO_FIRST, last = geo & GEO_LAST;
        // (rare) ordinary steps read the summaries from global memory
        const SumView S{A.smax, A.sarg, nullptr, nullptr, 0, 0, A.ssup};
        uint64_t v = first ? flo : st->entry_pos;
        uint64_t kb = excl, held = 0;
        uint32_t nb = 0;
        // lanes hold up to 32 pending boundaries; flushed as one coalesced store
        auto emit = [&](uint64_t val) {
            if ((uint32_t)lane == nb) held = val;
            if (++nb == 32) {
                if (kb + lane < A.capacity) A.out[kb + lane] = held;
                kb += 32;
                nb = 0;
            }
        };
        // one step the ordinary way (positions not on a logged chain)
        auto step = [&]() {
            const long long t_step = A.stats ? clock64() : 0;
            uint32_t k;
            uint64_t dd;
            const uint64_t e = w_advance<RULE>(S, R, P, flo - A.wctx, fhi, v, seg_hi, &k, &dd);
            if (lane == 0) stat_add(A, STAT_OUT_STEPS, 1);
            for (uint32_t i = 0; i < k; i++) {
                const uint64_t p = v + i * dd;
                if (p != flo) emit(p - flo);
            }
            v = e;
            if (A.stats && lane == 0) stat_add(A, STAT_CYC_OUT_STEPS, (unsigned long long)(clock64() - t_step));
        };
        const long long t_seg = clock64();
        if (!(geo & GEO_EMPTY)) {
            // the stitch kernel's walk from the entry, if it was logged: its
            // records run from the entry to the first speculated position
            const uint32_t es = first ? NONE : st->entry_slot;
            if (es < (uint32_t)NL && st->sw_cnt[es] != 0xFFFFu) {
                const uint32_t c = st->sw_cnt[es];
                const ulonglong2* sl = reinterpret_cast<const ulonglong2*>(A.plog) +
                                       item * (uint64_t)(A.logcap + SWCAP) + A.logcap + st->sw_first[es];
                static_assert(SWPW <= 64, "two records per lane");
                ulonglong2 r0 = make_ulonglong2(0, 0), r1 = make_ulonglong2(0, 0);
                if ((uint32_t)lane < c) r0 = sl[lane];
                if ((uint32_t)lane + 32 < c) r1 = sl[lane + 32];
                for (uint32_t i = 0; i < c; i++) {
                    const uint64_t p = __shfl_sync(FULL, i < 32 ? r0.x : r1.x, i & 31);
                    const uint64_t kd = __shfl_sync(FULL, i < 32 ? r0.y : r1.y, i & 31);
                    if (p != v) break;  // not the path from the entry: leave the rest to the loop below
                    const uint32_t k = (uint32_t)(kd >> 32);
                    const uint64_t d = (uint32_t)kd;
                    if (lane == 0) stat_add(A, STAT_OUT_RECS, 1);
                    for (uint32_t j = 0; j < k; j++) emit(v + j * d - flo);
                    v += (uint64_t)k * d;
                }
            }
            const uint32_t ln = st->log_n;
            const bool use_log = ln <= A.logcap;
            const unsigned long long* ht = A.hash + item * (uint64_t)HSTRIDE;
            const ulonglong2* lg = reinterpret_cast<const ulonglong2*>(A.plog) + item * (uint64_t)(A.logcap + SWCAP);
            constexpr uint64_t POS = (1ull << 57) - 1;
            while (v < seg_hi) {
                // the chain whose recorded path holds v (the first segment of a
                // file: chain 0 from the file start; it is never hashed)
                int m = -1;
                if (use_log) {
                    if (first) {
                        m = v == flo ? 0 : -1;
                    } else {
                        const uint32_t hv = hfind<RULE>(ht, (uint32_t)(v - seg_lo) + 1u);
                        m = hv == ~0u ? -1 : (int)(hv >> 16);
                    }
                }
                if (m < 0) {
                    step();
                    continue;
                }
                // replay chain m's records from v on, in log order (= path order)
                const uint64_t v_start = v;
                bool broken = false;
                if (lane == 0) stat_add(A, STAT_OUT_PASSES, 1);
                for (uint32_t b0 = 0; b0 < ln && !broken; b0 += 128) {
                    ulonglong2 r[4];
                    bool mine[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const uint32_t i = b0 + 32 * u + (uint32_t)lane;
                        mine[u] = false;
                        if (i < ln) {
                            r[u] = lg[i];
                            mine[u] = (uint32_t)(r[u].x >> 57) == (uint32_t)m && (r[u].x & POS) >= v_start;
                        } else {
                            r[u] = make_ulonglong2(0, 0);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        uint32_t bal = __ballot_sync(FULL, mine[u]);
                        while (bal && !broken) {
                            const int src = __ffs((int)bal) - 1;
                            bal &= bal - 1;
                            const uint64_t p = __shfl_sync(FULL, r[u].x, src) & POS;
                            const uint64_t kd = __shfl_sync(FULL, r[u].y, src);
                            if (p != v) {  // not the continuation of the path: leave it to ordinary steps
                                broken = true;
                                break;
                            }
                            const uint32_t k = (uint32_t)(kd >> 32);
                            const uint64_t d = (uint32_t)kd;
                            if (lane == 0) stat_add(A, STAT_OUT_RECS, 1);
                            for (uint32_t i = 0; i < k; i++) {
                                const uint64_t q = p + i * d;
                                if (q != flo) emit(q - flo);
                            }
                            v = p + (uint64_t)k * d;
                        }
                    }
                }
                if (v == v_start) step();  // no record continued the path
            }
            if (last) emit(fhi - flo);
        }
        if ((uint32_t)lane < nb && kb + lane < A.capacity) A.out[kb + lane] = held;
        kb += nb;
        if (lane == 0) stat_add(A, STAT_CYC_OUTPUT, (unsigned long long)(clock64() - t_seg));
        if (lane == 0) {
            if (kb - excl != cnt || (!first && !(geo & GEO_EMPTY) && st->entry_pos < seg_lo)) {
                atomicOr(&A.ctrl->err, ERR_INTERNAL);
                A.ctrl->err_info = item;
            }
            if (A.bounds_index && first) {
                const uint64_t f = A.item_file[item];
                A.bounds_index[f] = excl;
                for (uint64_t g2 = f; g2 > 0 && A.file_off[g2 - 1] == A.file_off[g2]; g2--)
                    A.bounds_index[g2 - 1] = excl;
            }
            if (A.bounds_index && item + 1 == n_items) {
                const uint64_t f = A.item_file[item];
                const uint64_t total = excl + cnt;
                A.bounds_index[A.n_files] = total;
                for (uint64_t g2 = A.n_files - 1; g2 > f && A.file_off[g2] == A.file_off[g2 + 1]; g2--)
                    A.bounds_index[g2] = total;
            }
        }
        __syncwarp();
    }
}

// ---- launchers --------------------------------------------------------------------------

int chain_smem(int rule, uint32_t win) {
    if (rule == RULE_RAM || rule == RULE_AE) return 2 * (int)win;
    if (rule == RULE_MAXP) return (int)win;
    return 16;
}

// Per-device memo of launch properties (function attributes set, occupancy),
// so that a call does not repeat those driver queries.
static std::mutex g_memo_mu;
struct Memo {
    int dev, key;
    uint32_t arg;
    int val;
};
static constexpr int kMemoCap = 512;
static Memo g_memo[kMemoCap];
static int g_memo_n = 0;

int launch_memo(int key, uint32_t arg, int (*fn)(uint32_t)) {
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(g_memo_mu);
        for (int i = 0; i < g_memo_n; i++)
            if (g_memo[i].dev == dev && g_memo[i].key == key && g_memo[i].arg == arg) return g_memo[i].val;
    }
    const int v = fn(arg);
    std::lock_guard<std::mutex> lock(g_memo_mu);
    if (g_memo_n < kMemoCap) g_memo[g_memo_n++] = Memo{dev, key, arg, v};
    return v;
}

template <int RULE>
int allow_smem() {
    return launch_memo(100 + RULE, 0, [](uint32_t) {
        int e = allow_max_smem(k_spec<RULE>);
        return e;
    });
}

template <int RULE>
static cudaError_t launch_rule(const ChainLaunch& a, const ChainGrids& gr, cudaStream_t st, int* launches,
                               cudaEvent_t ev_spec) {
    int sm = chain_smem(RULE, a.win);
    const int set = allow_smem<RULE>();
    if (set != (int)cudaSuccess) return (cudaError_t)set;
    k_spec<RULE><<<gr.spec, NL, sm, st>>>(a);
    if (ev_spec) cudaEventRecord(ev_spec, st);
    k_stitch<RULE><<<gr.stitch, NL, 0, st>>>(a);
    k_ures<RULE><<<gr.stitch, NL, 0, st>>>(a);
    k_compose<RULE><<<gr.groups, 32, 0, st>>>(a);
    k_scan<RULE><<<1, 32, 0, st>>>(a);
    k_settle<RULE><<<gr.groups, 32, 0, st>>>(a);
    k_output<RULE><<<gr.output, 32, 0, st>>>(a);
    *launches += 7;
    return cudaGetLastError();
}

cudaError_t launch_chain(const ChainLaunch& a, int rule, const ChainGrids& gr, cudaStream_t st, int* launches,
                         cudaEvent_t ev_spec) {
    switch (rule) {
    case RULE_RAM: return launch_rule<RULE_RAM>(a, gr, st, launches, ev_spec);
    case RULE_AE: return launch_rule<RULE_AE>(a, gr, st, launches, ev_spec);
    case RULE_MAXP: return launch_rule<RULE_MAXP>(a, gr, st, launches, ev_spec);
    case RULE_RAM_BYTES: return launch_rule<RULE_RAM_BYTES>(a, gr, st, launches, ev_spec);
    case RULE_AE_BYTES: return launch_rule<RULE_AE_BYTES>(a, gr, st, launches, ev_spec);
    default: return launch_rule<RULE_MAXP_BYTES>(a, gr, st, launches, ev_spec);
    }
}

template <int RULE>
static int occ_spec(uint32_t win) {
    allow_smem<RULE>();
    return launch_memo(200 + RULE, win, [](uint32_t wn) {
        int sm = chain_smem(RULE, wn), n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_spec<RULE>, NL, sm);
        return n > 0 ? n : 1;
    });
}

int spec_blocks_per_sm(int rule, uint32_t win) {
    switch (rule) {
    case RULE_RAM: return occ_spec<RULE_RAM>(win);
    case RULE_AE: return occ_spec<RULE_AE>(win);
    case RULE_MAXP: return occ_spec<RULE_MAXP>(win);
    case RULE_RAM_BYTES: return occ_spec<RULE_RAM_BYTES>(win);
    case RULE_AE_BYTES: return occ_spec<RULE_AE_BYTES>(win);
    default: return occ_spec<RULE_MAXP_BYTES>(win);
    }
}

}  // namespace cdc
