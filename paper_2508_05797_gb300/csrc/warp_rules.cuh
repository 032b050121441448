// warp_rules.cuh -- the chunk rules of chain_logic.cuh, executed by a whole
// warp for one chain (warp-uniform arguments and results).
//
// The per-thread rules make one thread follow one chain; when a single chain
// has to be followed (writing the boundaries, stitching a predecessor's exit,
// settling an uncovered entry) its latency is what matters. Here the 32 lanes
// share every scan: the Extreme Byte Search over a window takes 32 summary
// words (128 blocks = 8 KiB of input) per step and ends in __reduce_max_sync;
// the Range Scan compares 32 words at once and takes the first hit with a
// ballot -- the warp-level counterparts of the paper's tree-based search
// (Section 3.1) and packed scanning (Section 3.2). Results are identical to
// the per-thread rules (which the host tests check against the oracle).
#pragma once
#include "cdc_device.cuh"

namespace cdc {

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// max of m[] over blocks [b0, b1), b0 < b1
__device__ __forceinline__ uint32_t w_sum_max(const SumView& S, uint64_t b0, uint64_t b1) {
    const uint64_t we = (b1 + 3) >> 2;
    uint32_t acc = 0;
    for (uint64_t wi = (b0 >> 2) + lane_id(); wi < we; wi += 32) acc = vmax4(acc, clip_word(S.m4(wi), wi, b0, b1));
    return __reduce_max_sync(FULL, hmax4(acc));
}

// first block in [b0, b1) with m[] >= M (M >= 1); b1 if none
__device__ __forceinline__ uint64_t w_sum_first_geq(const SumView& S, uint64_t b0, uint64_t b1, uint32_t M) {
    const uint32_t Mx = M * 0x01010101u;
    const uint64_t we = (b1 + 3) >> 2;
    for (uint64_t base = b0 >> 2; base < we; base += 32) {
        const uint64_t wi = base + lane_id();
        uint32_t h = 0;
        if (wi < we) h = clip_word(vcmpge4(S.m4(wi), Mx), wi, b0, b1);
        const uint32_t bal = __ballot_sync(FULL, h != 0);
        if (bal) {
            const int l = __ffs((int)bal) - 1;
            const uint32_t hl = __shfl_sync(FULL, h, l);
            return ((base + (uint64_t)l) << 2) + (uint32_t)((ffs32(hl) - 1) >> 3);
        }
    }
    return b1;
}

// max byte of [a, b)
__device__ __forceinline__ uint32_t w_raw_max(const RawView& R, uint64_t a, uint64_t b) {
    const uint64_t we = (b + 3) >> 2;
    uint32_t acc = 0;
    for (uint64_t wi = (a >> 2) + lane_id(); wi < we; wi += 32) acc = vmax4(acc, clip_word(R.word(wi), wi, a, b));
    return __reduce_max_sync(FULL, hmax4(acc));
}

// first position in [a, b) with byte >= M (M >= 1); b if none
__device__ __forceinline__ uint64_t w_raw_first_geq(const RawView& R, uint64_t a, uint64_t b, uint32_t M,
                                                    uint32_t* val) {
    const uint32_t Mx = M * 0x01010101u;
    const uint64_t we = (b + 3) >> 2;
    for (uint64_t base = a >> 2; base < we; base += 32) {
        const uint64_t wi = base + lane_id();
        uint32_t v = 0, h = 0;
        if (wi < we) {
            v = R.word(wi);
            h = clip_word(vcmpge4(v, Mx), wi, a, b);
        }
        const uint32_t bal = __ballot_sync(FULL, h != 0);
        if (bal) {
            const int l = __ffs((int)bal) - 1;
            const uint32_t hl = __shfl_sync(FULL, h, l), vl = __shfl_sync(FULL, v, l);
            const uint32_t k = (uint32_t)((ffs32(hl) - 1) >> 3);
            *val = (vl >> (8 * k)) & 0xFFu;
            return ((base + (uint64_t)l) << 2) + k;
        }
    }
    return b;
}

// max of [a, b) and the first position holding it
__device__ __forceinline__ void w_raw_max_first(const RawView& R, uint64_t a, uint64_t b, uint32_t* v, uint64_t* p) {
    const uint32_t M = w_raw_max(R, a, b);
    uint32_t val;
    *p = M ? w_raw_first_geq(R, a, b, M, &val) : a;
    *v = M;
}

__device__ __forceinline__ uint32_t w_range_max(const SumView& S, const RawView& R, uint64_t a, uint64_t b) {
    const uint64_t ba = a >> 6, bl = (b - 1) >> 6;
    if (ba == bl) {
        if ((a & 63) == 0 && (b & 63) == 0) return S.m(ba);
        if (S.m(ba) == 0) return 0;
        return w_raw_max(R, a, b);
    }
    const uint64_t fb = (a + 63) >> 6, lb = b >> 6;
    uint32_t M = fb < lb ? w_sum_max(S, fb, lb) : 0;
    if ((a & 63) && S.m(ba) > M) {
        const uint32_t h = w_raw_max(R, a, (ba + 1) << 6);
        if (h > M) M = h;
    }
    if ((b & 63) && S.m(bl) > M) {
        const uint32_t t = w_raw_max(R, bl << 6, b);
        if (t > M) M = t;
    }
    return M;
}

__device__ __forceinline__ uint64_t w_first_geq(const SumView& S, const RawView& R, uint64_t from, uint64_t to,
                                                uint32_t M, uint32_t* val) {
    uint64_t b = from >> 6;
    const uint64_t bend = (to - 1) >> 6;
    if ((from & 63) != 0 || b == bend) {
        const uint64_t bhi = (b + 1) << 6;
        const uint32_t bm = S.m(b);
        if (bm >= M) {
            const uint64_t a = (b << 6) + S.a(b);
            if (bm == M && a >= from) {
                if (a < to) { *val = M; return a; }
                return to;
            }
            const uint64_t e = umin64(bhi, to);
            const uint64_t r = w_raw_first_geq(R, from, e, M, val);
            if (r < e) return r;
        }
        if (b == bend) return to;
        b++;
    }
    while (b <= bend) {
        const uint64_t bh = w_sum_first_geq(S, b, bend + 1, M);
        if (bh > bend) return to;
        const uint64_t blo = bh << 6;
        const uint32_t bm = S.m(bh);
        const uint64_t a = blo + S.a(bh);
        if (bm == M) {
            if (a < to) { *val = M; return a; }
            return to;
        }
        const uint64_t e = umin64(blo + 64, to);
        const uint64_t r = w_raw_first_geq(R, blo, e, M, val);
        if (r < e) return r;
        if (e == to) return to;
        b = bh + 1;
    }
    return to;
}

__device__ __forceinline__ uint64_t w_next_ram(const SumView& S, const RawView& R, const Prm& P, uint64_t fhi,
                                               uint64_t s) {
    if (fhi - s <= P.w) return fhi;
    const uint64_t limit = umin64(fhi, s + P.mx);
    const uint64_t t = s + P.w;
    const uint32_t M = w_range_max(S, R, s, t);
    const uint64_t j0 = umax64(t, s + P.mn - 1);
    if (j0 >= limit) return limit;
    if (M == 0) return j0 + 1;
    uint32_t val;
    const uint64_t j = w_first_geq(S, R, j0, limit, M, &val);
    return j < limit ? j + 1 : limit;
}

__device__ __forceinline__ uint64_t w_next_ae(const SumView& S, const RawView& R, const Prm& P, uint64_t fhi,
                                              uint64_t s) {
    const uint64_t limit = umin64(fhi, s + P.mx);
    if (s + 1 >= limit) return limit;
    uint64_t p;
    uint32_t v;
    {
        const uint64_t b = s >> 6;
        const uint64_t a = (b << 6) + S.a(b);
        if (a >= s && a < limit) {
            p = a;
            v = S.m(b);
        } else {
            w_raw_max_first(R, s, umin64((b + 1) << 6, limit), &v, &p);
        }
    }
    uint64_t cur = p + 1;
    for (;;) {
        const uint64_t t = umax64(p + P.w, s + P.mn - 1);
        if (t >= limit) return limit;
        if (v == 255) return t + 1;
        const uint64_t to = t + 1;
        if (cur & 63) {
            const uint64_t bc = cur >> 6, bhi = (bc + 1) << 6;
            const uint32_t bm = S.m(bc);
            if (bm > v) {
                const uint64_t a = (bc << 6) + S.a(bc);
                if (a >= cur && bhi <= to) {
                    p = a; v = bm; cur = a + 1;
                    continue;
                }
                const uint64_t e = umin64(bhi, to);
                uint32_t val;
                const uint64_t q = w_raw_first_geq(R, cur, e, v + 1, &val);
                if (q < e) {
                    p = q; v = val; cur = q + 1;
                    continue;
                }
            }
            if (bhi >= to) return to;
            cur = bhi;
        }
        const uint64_t bf = cur >> 6, bl = (to - 1) >> 6;
        const uint64_t bh = w_sum_first_geq(S, bf, bl + 1, v + 1);
        if (bh > bl) return to;
        const uint64_t blo = bh << 6;
        if (blo + 64 <= to) {
            p = blo + S.a(bh); v = S.m(bh); cur = p + 1;
            continue;
        }
        uint32_t val;
        const uint64_t q = w_raw_first_geq(R, blo, to, v + 1, &val);
        if (q < to) {
            p = q; v = val; cur = q + 1;
            continue;
        }
        return to;
    }
}

// first block in [b0, b1) holding a MAXP target >= cmin and < cend; returns the target or cend
__device__ __forceinline__ uint64_t w_next_maxp(const SumView& S, const Prm& P, uint64_t flo, uint64_t fhi,
                                                uint64_t s) {
    const uint64_t limit = umin64(fhi, s + P.mx);
    const uint64_t cmin = umax64(s + P.mn - 1, flo + P.w);
    const uint64_t cend = fhi > flo + P.w ? umin64(limit, fhi - P.w) : 0;
    if (cmin >= cend) return limit;
    const uint64_t b0 = cmin >> 6, b1 = ((cend - 1) >> 6) + 1, we = (b1 + 3) >> 2;
    for (uint64_t base = b0 >> 2; base < we; base += 32) {
        const uint64_t wi = base + lane_id();
        uint64_t c = ~0ull;
        if (wi < we) {
            const uint32_t v = S.m4(wi);
            if (v != 0xFFFFFFFFu) {
#pragma unroll
                for (int k = 3; k >= 0; k--) {  // keep the smallest valid target of the word
                    const uint64_t bb = (wi << 2) + k;
                    const uint32_t o = (v >> (8 * k)) & 0xFFu;
                    if (o == 0xFFu || bb < b0 || bb >= b1) continue;
                    const uint64_t cc = (bb << 6) + o;
                    if (cc >= cmin && cc < cend) c = cc;
                }
            }
        }
        const uint32_t bal = __ballot_sync(FULL, c != ~0ull);
        if (bal) return __shfl_sync(FULL, c, __ffs((int)bal) - 1) + 1;
    }
    return limit;
}

// first non-zero byte in [p, bound), skipping quiet superblocks: lanes test
// 32 superblocks (or 32 blocks) at a time
__device__ __forceinline__ uint64_t w_first_nonzero(const SumView& S, const RawView& R, uint64_t p, uint64_t bound) {
    while (p < bound) {
        if ((p & 4095) == 0 && S.sup && p + 4096 <= bound) {
            // superblocks [p>>12, ...) wholly below bound
            const uint64_t q0 = p >> 12, qn = (bound >> 12) - q0;
            const uint64_t q = q0 + lane_id();
            const bool loud = (uint64_t)lane_id() < qn && S.sup[q] != 0;
            const uint32_t bal = __ballot_sync(FULL, loud);
            if (bal == 0 && qn >= 32) { p += 32ull << 12; continue; }
            if (bal == 0) { p = (q0 + qn) << 12; continue; }
            const int l = __ffs((int)bal) - 1;
            if (l > 0) { p = (q0 + (uint64_t)l) << 12; continue; }
        }
        // blocks from p up to the next superblock boundary (or bound)
        const uint64_t e = umin64(bound, ((p >> 12) + 1) << 12);
        const uint64_t b0 = p >> 6, b1 = ((e - 1) >> 6) + 1;
        const uint64_t bb = b0 + lane_id();
        const bool nz = bb < b1 && S.m(bb) != 0;
        const uint32_t bal = __ballot_sync(FULL, nz);
        if (bal == 0) {
            p = umin64(e, (b0 + 32) << 6);
            continue;
        }
        const uint64_t hb = b0 + (uint64_t)(__ffs((int)bal) - 1);
        const uint64_t lo = umax64(p, hb << 6), hi = umin64(bound, (hb + 1) << 6);
        uint32_t val;
        const uint64_t r = w_raw_first_geq(R, lo, hi, 1, &val);
        if (r < hi) return r;
        p = hi;
    }
    return bound;
}

// first MAXP target in [c0, c1), skipping superblocks without one
__device__ __forceinline__ uint64_t w_first_target(const SumView& S, uint64_t c0, uint64_t c1) {
    uint64_t p = c0;
    while (p < c1) {
        if ((p & 4095) == 0 && S.sup && p + 4096 <= c1) {
            const uint64_t q0 = p >> 12, qn = (c1 >> 12) - q0;
            const bool has = (uint64_t)lane_id() < qn && S.sup[q0 + lane_id()] != 0;
            const uint32_t bal = __ballot_sync(FULL, has);
            if (bal == 0) { p = (q0 + umin64(qn, 32)) << 12; continue; }
            const int l = __ffs((int)bal) - 1;
            if (l > 0) { p = (q0 + (uint64_t)l) << 12; continue; }
        }
        const uint64_t e = umin64(c1, ((p >> 12) + 1) << 12);
        const uint64_t b0 = p >> 6, b1 = ((e - 1) >> 6) + 1;
        const uint64_t bb = b0 + lane_id();
        uint64_t c = ~0ull;
        if (bb < b1) {
            const uint32_t o = S.m(bb);
            if (o != 0xFFu) {
                const uint64_t cc = (bb << 6) + o;
                if (cc >= p && cc < c1) c = cc;
            }
        }
        const uint32_t bal = __ballot_sync(FULL, c != ~0ull);
        if (bal) return __shfl_sync(FULL, c, __ffs((int)bal) - 1);
        p = umin64(e, (b0 + 32) << 6);
    }
    return c1;
}

template <int RULE>
__device__ __forceinline__ uint64_t w_next(const SumView& S, const RawView& R, const Prm& P, uint64_t flo,
                                           uint64_t fhi, uint64_t s) {
    if (RULE == RULE_RAM) return w_next_ram(S, R, P, fhi, s);
    if (RULE == RULE_AE) return w_next_ae(S, R, P, fhi, s);
    if (RULE == RULE_MAXP) return w_next_maxp(S, P, flo, fhi, s);
    return next_cut<RULE>(S, R, P, flo, fhi, s);  // byte rules: every lane runs the same steps
}

// warp version of advance(): same contract (k steps of stride d, then e)
template <int RULE>
__device__ __forceinline__ uint64_t w_advance(const SumView& S, const RawView& R, const Prm& P, uint64_t flo,
                                              uint64_t fhi, uint64_t s, uint64_t stop, uint32_t* k, uint64_t* d) {
    if (RULE == RULE_RAM || RULE == RULE_AE) {
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
    }
    if (RULE == RULE_MAXP) {
        const uint64_t e1 = w_next_maxp(S, P, flo, fhi, s);
        if (e1 == s + P.mx && e1 < fhi) {
            const uint64_t mx = P.mx;
            const uint64_t c0 = umax64(s + P.mn - 1, flo + P.w);
            const uint64_t cend = fhi > flo + P.w ? fhi - P.w : 0;
            const uint64_t kstop = (stop - 1 - s) / mx + 1;
            const uint64_t kfhi = (fhi - s) / mx;
            const uint64_t kmax = kstop < kfhi ? kstop : kfhi;
            if (kmax >= 2) {
                const uint64_t lim = umin64(cend, s + kmax * mx);
                const uint64_t c = c0 < lim ? w_first_target(S, c0, lim) : lim;
                const uint64_t kc = c >= s + mx ? (c - s - mx) / mx + 1 : 0;
                const uint64_t kk = kc < kmax ? kc : kmax;
                if (kk >= 2) {
                    *k = (uint32_t)kk;
                    *d = mx;
                    return s + kk * mx;
                }
            }
        }
        *k = 1;
        *d = e1 - s;
        return e1;
    }
    const uint64_t e = w_next<RULE>(S, R, P, flo, fhi, s);
    *k = 1;
    *d = e - s;
    return e;
}

}  // namespace cdc
