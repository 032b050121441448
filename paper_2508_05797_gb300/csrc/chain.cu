// chain.cu -- stage 2: the chunk chain, in parallel and bit-exact.
//
// Each chunk starts where the previous one ended, so the chunk starts form a
// single chain s_{i+1} = next(s_i) (Section 3.3: every algorithm is a loop of
// extreme byte searches and range scans over one chunk at a time). Chains
// started at different offsets join only where their cuts coincide, and for
// RAM and AE on random bytes that can take hundreds of kilobytes, so a single
// speculative chain per segment would almost never line up with the true
// one. The stage therefore works per segment ("item") of the input, one warp
// per item, in four steps:
//
//  A. Speculate: each of the 32 lanes runs its own chain (per-thread next())
//     from a different start spread over the first `span` bytes of the
//     segment, recording its first KFIRST positions, its count and its exit
//     (first position at or past the segment end).
//  B. Stitch: for every distinct exit of the previous segment's 32 chains,
//     the warp follows the chain from that exit until it lands on a recorded
//     position of one of this segment's lanes (or reaches the segment end and
//     matches a lane's exit). The result is a 32-entry table: predecessor
//     chain -> (this segment's chain, number of boundaries in the segment).
//  C. Resolve: decoupled look-back. Find the nearest earlier segment whose
//     true state is published, then carry that state forward through the
//     tables of the segments in between (warp shuffles), publishing each
//     segment's true state on the way so that later warps start closer.
//     Entries the tables do not cover are settled by following the chain
//     through that segment directly.
//  D. Output: follow the true chain through the segment once more and write
//     its boundaries at the global offset found in C.
//
// All waits are bounded (globaltimer); on expiry the kernel records
// ERR_TIMEOUT in the control block and every warp leaves.
#include "cdc_device.cuh"
#include "cdc_launch.h"

namespace cdc {

struct Lanes {
    uint32_t fp[KFIRST];  // first positions of this lane's chain (offsets from seg_lo)
    uint32_t c;           // positions of the chain inside the segment
    uint64_t x;           // exit of the chain
};

struct WalkResult {
    uint32_t code;   // tab_enc(slot, count), or TAB_UNKNOWN when no chain was joined
    uint64_t exit;   // exit position of the followed chain
    uint32_t count;  // boundaries inside the segment
};

// Follow the chain from entry e through [seg_lo, seg_hi) until it joins one
// of the segment's 32 chains. Warp-uniform: every lane computes the same
// steps; lane l tests membership in its own chain.
template <int RULE>
__device__ WalkResult walk(const SumView& S, const RawView& R, const Prm& P, uint64_t flo, uint64_t fhi,
                           uint64_t seg_lo, uint64_t seg_hi, bool last, const Lanes& L, uint64_t e) {
    uint64_t v = e;
    uint32_t ne = 0;
    while (v < seg_hi) {
        int idx = -1;
#pragma unroll
        for (int t = KFIRST - 1; t >= 0; t--)
            if ((uint32_t)t < L.c && seg_lo + L.fp[t] == v) idx = t;
        uint32_t hm = __ballot_sync(FULL, idx >= 0);
        if (hm) {
            int m = __ffs((int)hm) - 1;
            int im = __shfl_sync(FULL, idx, m);
            uint32_t cm = __shfl_sync(FULL, L.c, m);
            uint64_t xm = __shfl_sync(FULL, L.x, m);
            uint32_t cnt = ne + cm - (uint32_t)im + (last ? 1u : 0u);
            return {tab_enc((uint32_t)m, cnt), xm, cnt};
        }
        v = next_cut<RULE>(S, R, P, flo, fhi, v);
        ne++;
    }
    uint32_t cnt = ne + (last ? 1u : 0u);
    uint32_t xm = __ballot_sync(FULL, L.x == v);
    if (xm) return {tab_enc((uint32_t)(__ffs((int)xm) - 1), cnt), v, cnt};
    return {TAB_UNKNOWN, v, cnt};
}

// lane 0 waits (bounded) until *f == epoch; false on timeout or error
__device__ bool wait_flag(const unsigned int* f, uint32_t epoch, const ChainLaunch& A, uint64_t item) {
    uint32_t ok = 1;
    if ((threadIdx.x & 31) == 0 && ld_acquire(f) != epoch) {
        uint64_t t0 = gtimer_ns();
        for (;;) {
            if (ld_acquire(f) == epoch) break;
            if (ld_volatile(&A.ctrl->err)) { ok = 0; break; }
            if (gtimer_ns() - t0 > A.timeout_ns) {
                atomicOr(&A.ctrl->err, ERR_TIMEOUT);
                A.ctrl->err_info = item;
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
    }
    ok = __shfl_sync(FULL, ok, 0);
    __syncwarp();
    return ok != 0;
}

__device__ __forceinline__ void publish_final(ItemStatus* it, uint32_t slot, uint64_t exit, uint64_t incl,
                                              uint32_t epoch) {
    if (ld_acquire(&it->flagFIN) == epoch) return;
    it->fin_slot = slot;
    it->fin_exit = exit;
    it->fin_incl = incl;
    __threadfence();
    st_release(&it->flagFIN, epoch);
}

// True state after segment jt: the chain's slot in jt (or NONE_SLOT), its exit
// position and the number of boundaries up to and including jt.
template <int RULE>
__device__ bool resolve(const ChainLaunch& A, uint32_t epoch, uint64_t jt, const Prm& P, const RawView& R,
                        uint32_t* o_slot, uint64_t* o_pos, uint64_t* o_incl) {
    const int lane = threadIdx.x & 31;
    // 1) nearest segment with a published true state; every later one up to
    //    jt must have published its table
    int64_t j = -1;
    uint64_t t0 = 0;
    bool timing = false;
    for (;;) {
        int64_t base = (int64_t)jt;
        for (;;) {
            int64_t i = base - lane;
            bool valid = i >= 0;
            uint32_t ff = valid ? ld_acquire(&A.st[i].flagFIN) : 0u;
            uint32_t fa = valid ? ld_acquire(&A.st[i].flagAGG) : 0u;
            uint32_t fm = __ballot_sync(FULL, valid && ff == epoch);
            uint32_t am = __ballot_sync(FULL, !valid || ff == epoch || fa == epoch);
            if (fm) {
                int l = __ffs((int)fm) - 1;
                uint32_t need = l ? ((1u << l) - 1u) : 0u;
                if ((am & need) == need) j = base - l;
                break;
            }
            if (am != FULL || base < 32) break;
            base -= 32;
        }
        if (j >= 0) break;
        uint32_t bad = 0;
        if (lane == 0) {
            if (!timing) { t0 = gtimer_ns(); timing = true; }
            if (ld_volatile(&A.ctrl->err)) bad = 1;
            else if (gtimer_ns() - t0 > A.timeout_ns) {
                atomicOr(&A.ctrl->err, ERR_TIMEOUT);
                A.ctrl->err_info = jt;
                bad = 1;
            }
            __nanosleep(128);
        }
        if (__shfl_sync(FULL, bad, 0)) return false;
    }
    __syncwarp();
    uint32_t slot = A.st[j].fin_slot;
    uint64_t pos = A.st[j].fin_exit;
    uint64_t incl = A.st[j].fin_incl;
    // 2) carry the state forward, 8 segments per round
    const SumView Sg{A.smax, A.sarg, nullptr, nullptr, 0, 0};
    uint64_t i = (uint64_t)j + 1;
    while (i <= jt) {
        const uint32_t nbat = (uint32_t)umin64(8, jt - i + 1);
        uint32_t tb[8];
#pragma unroll
        for (int t = 0; t < 8; t++) tb[t] = (uint32_t)t < nbat ? A.st[i + t].table[lane] : 0u;
        uint32_t done = 0, my_sl = 0, my_cn = 0;
#pragma unroll
        for (int t = 0; t < 8; t++) {
            if ((uint32_t)t < nbat && done == (uint32_t)t) {
                uint32_t e0 = __shfl_sync(FULL, tb[t], 0);
                uint32_t e = (e0 & TAB_CONST) ? e0 : (slot < 32 ? __shfl_sync(FULL, tb[t], (int)slot) : TAB_UNKNOWN);
                if (!(e & TAB_UNKNOWN)) {
                    slot = tab_slot(e);
                    if (lane == t) { my_sl = slot; my_cn = tab_count(e); }
                    done++;
                }
            }
        }
        if (done) {
            uint64_t my_pos = 0;
            if ((uint32_t)lane < done) my_pos = A.st[i + lane].X[my_sl];
            uint64_t c64 = (uint32_t)lane < done ? my_cn : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                uint64_t o = __shfl_up_sync(FULL, c64, d);
                if (lane >= d) c64 += o;
            }
            uint64_t my_incl = incl + c64;
            if ((uint32_t)lane < done && (int64_t)(i + lane) != A.hold_item)
                publish_final(&A.st[i + lane], my_sl, my_pos, my_incl, epoch);
            pos = __shfl_sync(FULL, my_pos, (int)done - 1);
            incl = __shfl_sync(FULL, my_incl, (int)done - 1);
            i += done;
        }
        if (done < nbat) {
            // segment i does not cover this entry: follow the chain through it
            ItemStatus* it = &A.st[i];
            Lanes L;
#pragma unroll
            for (int t = 0; t < KFIRST; t++) L.fp[t] = it->first[lane][t];
            L.c = it->cnt[lane];
            L.x = it->X[lane];
            const uint64_t s_lo = it->seg_lo, s_hi = it->seg_hi, flo = it->flo, fhi = it->fhi;
            const bool last = (it->geo & 2u) != 0;
            WalkResult r = walk<RULE>(Sg, R, P, flo, fhi, s_lo, s_hi, last, L, pos);
            slot = (r.code & TAB_UNKNOWN) ? NONE_SLOT : tab_slot(r.code);
            pos = r.exit;
            incl += r.count;
            if (lane == 0 && (int64_t)i != A.hold_item) publish_final(it, slot, pos, incl, epoch);
            i++;
        }
    }
    *o_slot = slot;
    *o_pos = pos;
    *o_incl = incl;
    return true;
}

template <int RULE>
__device__ bool process(const ChainLaunch& A, uint64_t item, uint32_t epoch, uint8_t* smem) {
    const int lane = threadIdx.x & 31;
    // ---- geometry
    uint64_t f, flo_l, fhi_l, kin;
    if (A.file_off == nullptr) {
        f = 0; flo_l = 0; fhi_l = A.single_len; kin = item;
    } else {
        f = A.item_file[item];
        flo_l = A.file_off[f];
        fhi_l = A.file_off[f + 1];
        kin = item - A.item_off[f];
    }
    const uint64_t flo = A.lo + flo_l, fhi = A.lo + fhi_l;
    const uint64_t seg_lo = flo + kin * A.seg;
    const uint64_t seg_hi = umin64(seg_lo + A.seg, fhi);
    const bool first = kin == 0, last = seg_hi == fhi;
    ItemStatus* me = &A.st[item];
    const bool hold = (int64_t)item == A.hold_item;
    const Prm P{A.w, A.mn, A.mx};
    const RawView R{A.base, A.inv};

    // ---- stage this segment's summaries in shared memory
    SumView S{A.smax, A.sarg, smem, smem + A.win, 0, 0};
    if (RULE == RULE_RAM || RULE == RULE_AE || RULE == RULE_MAXP) {
        uint64_t wb0 = (seg_lo >> 6) & ~15ull;
        uint64_t wn = A.win;
        if (wb0 + wn > A.nblk_pad) wn = A.nblk_pad > wb0 ? ((A.nblk_pad - wb0) & ~15ull) : 0;
        for (uint64_t o = (uint64_t)lane * 16; o < wn; o += 512) {
            *reinterpret_cast<uint4*>(smem + o) = *reinterpret_cast<const uint4*>(A.smax + wb0 + o);
            if (RULE != RULE_MAXP)
                *reinterpret_cast<uint4*>(smem + A.win + o) = *reinterpret_cast<const uint4*>(A.sarg + wb0 + o);
        }
        S.wb0 = wb0;
        S.wn = wn;
        __syncwarp();
    }

    // ---- A: 32 speculative chains
    Lanes L;
#pragma unroll
    for (int t = 0; t < KFIRST; t++) L.fp[t] = 0;
    L.c = 0;
    L.x = ~0ull;
    {
        uint64_t start = ~0ull;
        if (first) {
            if (lane == 0) start = flo;
        } else {
            uint64_t len = seg_hi - seg_lo;
            uint64_t d = umin64(A.span, len) / 32;
            if (d == 0) d = 1;
            start = seg_lo + (uint64_t)lane * d;
        }
        if (start < seg_hi) {
            uint64_t s = start;
            uint32_t c = 0;
            while (s < seg_hi) {
#pragma unroll
                for (int t = 0; t < KFIRST; t++)
                    if ((uint32_t)t == c) L.fp[t] = (uint32_t)(s - seg_lo);
                c++;
                s = next_cut<RULE>(S, R, P, flo, fhi, s);
            }
            L.c = c;
            L.x = s;
        }
    }
    me->X[lane] = L.x;
#pragma unroll
    for (int t = 0; t < KFIRST; t++) me->first[lane][t] = L.fp[t];
    me->cnt[lane] = L.c;
    if (lane == 0) {
        me->seg_lo = seg_lo;
        me->seg_hi = seg_hi;
        me->flo = flo;
        me->fhi = fhi;
        me->geo = (first ? 1u : 0u) | (last ? 2u : 0u);
    }
    __syncwarp();
    __threadfence();
    if (lane == 0 && !hold) st_release(&me->flagA, epoch);

    // ---- B: stitching table
    uint32_t tab = TAB_UNKNOWN;
    if (first) {
        uint32_t c0 = __shfl_sync(FULL, L.c, 0);
        tab = tab_enc(0, c0 - 1 + (last ? 1u : 0u)) | TAB_CONST;
    } else {
        if (!wait_flag(&A.st[item - 1].flagA, epoch, A, item)) return false;
        const uint64_t xp = A.st[item - 1].X[lane];
        uint32_t todo = __ballot_sync(FULL, xp != ~0ull);
        while (todo) {
            const int ld = __ffs((int)todo) - 1;
            const uint64_t e = __shfl_sync(FULL, xp, ld);
            const uint32_t same = __ballot_sync(FULL, xp == e) & todo;
            WalkResult r = walk<RULE>(S, R, P, flo, fhi, seg_lo, seg_hi, last, L, e);
            if ((same >> lane) & 1u) tab = r.code;
            todo &= ~same;
        }
    }
    me->table[lane] = tab;
    __syncwarp();
    __threadfence();
    if (lane == 0 && !hold) st_release(&me->flagAGG, epoch);

    // ---- C: true entry and global offset
    uint32_t eslot = NONE_SLOT;
    uint64_t epos = flo, excl = 0;
    if (item > 0 && !resolve<RULE>(A, epoch, item - 1, P, R, &eslot, &epos, &excl)) return false;
    uint32_t mslot;
    uint64_t mexit;
    uint32_t mcnt;
    if (first) {
        mslot = 0;
        mexit = __shfl_sync(FULL, L.x, 0);
        mcnt = tab_count(tab);
    } else {
        uint32_t e = eslot < 32 ? __shfl_sync(FULL, tab, (int)eslot) : TAB_UNKNOWN;
        if (!(e & TAB_UNKNOWN)) {
            mslot = tab_slot(e);
            mcnt = tab_count(e);
            mexit = __shfl_sync(FULL, L.x, (int)mslot);
        } else {
            WalkResult r = walk<RULE>(S, R, P, flo, fhi, seg_lo, seg_hi, last, L, epos);
            mslot = (r.code & TAB_UNKNOWN) ? NONE_SLOT : tab_slot(r.code);
            mexit = r.exit;
            mcnt = r.count;
        }
    }
    if (lane == 0 && !hold) publish_final(me, mslot, mexit, excl + mcnt, epoch);

    // ---- D: write the boundaries of the true chain
    {
        uint64_t v = first ? flo : epos;
        uint64_t kb = excl;
        uint64_t held = 0;
        uint32_t nb = 0;
        while (v < seg_hi) {
            if (v != flo) {
                if ((uint32_t)lane == nb) held = v - flo;
                if (++nb == 32) {
                    if (kb + lane < A.capacity) A.out[kb + lane] = held;
                    kb += 32;
                    nb = 0;
                }
            }
            v = next_cut<RULE>(S, R, P, flo, fhi, v);
        }
        if (last) {
            if ((uint32_t)lane == nb) held = fhi - flo;
            nb++;
        }
        if ((uint32_t)lane < nb && kb + lane < A.capacity) A.out[kb + lane] = held;
        kb += nb;
        if (kb - excl != mcnt || (!first && epos < seg_lo)) {
            if (lane == 0) {
                atomicOr(&A.ctrl->err, ERR_INTERNAL);
                A.ctrl->err_info = item;
            }
        }
    }

    // ---- per-file offsets and the total
    if (lane == 0) {
        if (A.bounds_index && first) {
            A.bounds_index[f] = excl;
            for (uint64_t g = f; g > 0 && A.file_off[g - 1] == A.file_off[g]; g--) A.bounds_index[g - 1] = excl;
        }
        const uint64_t n_items = A.n_items_dev ? *A.n_items_dev : A.n_items;
        if (item + 1 == n_items) {
            const uint64_t total = excl + mcnt;
            A.ctrl->total = total;
            if (A.d_count) *A.d_count = total;
            if (A.bounds_index) {
                A.bounds_index[A.n_files] = total;
                for (uint64_t g = A.n_files - 1; g > f && A.file_off[g] == A.file_off[g + 1]; g--)
                    A.bounds_index[g] = total;
            }
        }
    }
    __syncwarp();
    return true;
}

template <int RULE>
__global__ void __launch_bounds__(32) k_chain(ChainLaunch A) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const uint32_t epoch = ld_volatile(&A.ctrl->epoch);
    const uint64_t n_items =
        A.n_items_dev ? *reinterpret_cast<const volatile unsigned long long*>(A.n_items_dev) : A.n_items;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(&A.ctrl->ticket, 1ull);
        item = __shfl_sync(FULL, item, 0);
        if (item >= n_items) break;
        if (ld_volatile(&A.ctrl->err)) break;
        if (!process<RULE>(A, item, epoch, smem)) break;
    }
}

int chain_smem(int rule, uint32_t win) {
    if (rule == RULE_RAM || rule == RULE_AE) return 2 * (int)win;
    if (rule == RULE_MAXP) return (int)win;
    return 16;
}

template <int RULE>
static cudaError_t launch_rule(const ChainLaunch& a, int grid, cudaStream_t st) {
    int sm = chain_smem(RULE, a.win);
    cudaError_t e = cudaFuncSetAttribute(k_chain<RULE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    k_chain<RULE><<<grid, 32, sm, st>>>(a);
    return cudaGetLastError();
}

template <int RULE>
static int occupancy_rule(uint32_t win) {
    int sm = chain_smem(RULE, win), n = 0;
    cudaFuncSetAttribute(k_chain<RULE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_chain<RULE>, 32, sm);
    return n > 0 ? n : 1;
}

cudaError_t launch_chain(const ChainLaunch& a, int rule, int grid, cudaStream_t st) {
    switch (rule) {
    case RULE_RAM: return launch_rule<RULE_RAM>(a, grid, st);
    case RULE_AE: return launch_rule<RULE_AE>(a, grid, st);
    case RULE_MAXP: return launch_rule<RULE_MAXP>(a, grid, st);
    case RULE_RAM_BYTES: return launch_rule<RULE_RAM_BYTES>(a, grid, st);
    case RULE_AE_BYTES: return launch_rule<RULE_AE_BYTES>(a, grid, st);
    default: return launch_rule<RULE_MAXP_BYTES>(a, grid, st);
    }
}

int chain_blocks_per_sm(int rule, uint32_t win) {
    switch (rule) {
    case RULE_RAM: return occupancy_rule<RULE_RAM>(win);
    case RULE_AE: return occupancy_rule<RULE_AE>(win);
    case RULE_MAXP: return occupancy_rule<RULE_MAXP>(win);
    case RULE_RAM_BYTES: return occupancy_rule<RULE_RAM_BYTES>(win);
    case RULE_AE_BYTES: return occupancy_rule<RULE_AE_BYTES>(win);
    default: return occupancy_rule<RULE_MAXP_BYTES>(win);
    }
}

}  // namespace cdc
