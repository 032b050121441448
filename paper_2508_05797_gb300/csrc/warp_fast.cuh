// warp_fast.cuh -- the whole-warp chain rules of warp_rules.cuh for steps whose
// every access lies inside a segment's staged summary window.
//
// A speculative chain spends almost all of its steps inside the window the
// speculation kernel stages in shared memory. There a step can work on 32-bit
// offsets from the window start instead of 64-bit positions, read summaries
// straight from shared memory without a window test per access, and compare
// bytes in 16-bit lanes (ByteMax, ge_flags) instead of emulated byte-SIMD
// instructions. f_advance() takes that path when the step provably stays in
// the window and otherwise calls w_advance(); both give the same result (the
// GPU parity tests exercise both).
#pragma once
#include "warp_rules.cuh"

namespace cdc {

// A staged window: m[] (and a[] for RAM/AE) of the blocks covering bytes
// [p0, p0 + nb), in shared memory. p0 is a multiple of 1024.
struct Win {
    const uint8_t* m;
    const uint8_t* a;
    uint64_t p0;
    uint32_t nb;
};

// keep the bytes of word wi (units [4wi, 4wi + 4)) that lie in [a, b)
__device__ __forceinline__ uint32_t f_clip(uint32_t v, uint32_t wi, uint32_t a, uint32_t b) {
    const uint32_t lo = wi << 2;
    if (lo + 4 <= a || lo >= b) return 0;
    if (lo < a) v &= 0xFFFFFFFFu << (8 * (a - lo));
    if (lo + 4 > b) v &= 0xFFFFFFFFu >> (8 * (lo + 4 - b));
    return v;
}

__device__ __forceinline__ uint32_t f_m4(const Win& W, uint32_t wi) {
    return *reinterpret_cast<const uint32_t*>(W.m + 4 * wi);
}

// max of m[] over window blocks [b0, b1), b0 < b1
__device__ __forceinline__ uint32_t f_sum_max(const Win& W, uint32_t b0, uint32_t b1) {
    const uint32_t we = (b1 + 3) >> 2;
    ByteMax m;
    for (uint32_t wi = (b0 >> 2) + lane_id(); wi < we; wi += 32) m.add(f_clip(f_m4(W, wi), wi, b0, b1));
    return __reduce_max_sync(FULL, m.get());
}

// first window block in [b0, b1) with m[] >= M (M >= 1); b1 if none
__device__ __forceinline__ uint32_t f_sum_first_geq(const Win& W, uint32_t b0, uint32_t b1, uint32_t M) {
    const uint32_t K = ge_key(M), we = (b1 + 3) >> 2;
    for (uint32_t base = b0 >> 2; base < we; base += 32) {
        const uint32_t wi = base + lane_id();
        uint32_t f = 0;
        if (wi < we) f = ge_flags(f_clip(f_m4(W, wi), wi, b0, b1), K);
        const uint32_t bal = __ballot_sync(FULL, f != 0);
        if (bal) {
            const int l = __ffs((int)bal) - 1;
            const uint32_t fl = __shfl_sync(FULL, f, l);
            return ((base + (uint32_t)l) << 2) + (uint32_t)((__ffs((int)fl) - 1) >> 3);
        }
    }
    return b1;
}

// max byte of window bytes [a, b)
__device__ __forceinline__ uint32_t f_raw_max(const Win& W, const RawView& R, uint32_t a, uint32_t b) {
    const uint64_t gw0 = W.p0 >> 2;
    const uint32_t we = (b + 3) >> 2;
    ByteMax m;
    for (uint32_t wi = (a >> 2) + lane_id(); wi < we; wi += 32) m.add(f_clip(R.word(gw0 + wi), wi, a, b));
    return __reduce_max_sync(FULL, m.get());
}

// first window byte in [a, b) that is >= M (M >= 1); b if none
__device__ __forceinline__ uint32_t f_raw_first_geq(const Win& W, const RawView& R, uint32_t a, uint32_t b, uint32_t M,
                                                    uint32_t* val) {
    const uint64_t gw0 = W.p0 >> 2;
    const uint32_t K = ge_key(M), we = (b + 3) >> 2;
    for (uint32_t base = a >> 2; base < we; base += 32) {
        const uint32_t wi = base + lane_id();
        uint32_t v = 0, f = 0;
        if (wi < we) {
            v = R.word(gw0 + wi);
            f = ge_flags(f_clip(v, wi, a, b), K);
        }
        const uint32_t bal = __ballot_sync(FULL, f != 0);
        if (bal) {
            const int l = __ffs((int)bal) - 1;
            const uint32_t fl = __shfl_sync(FULL, f, l), vl = __shfl_sync(FULL, v, l);
            const uint32_t k = (uint32_t)((__ffs((int)fl) - 1) >> 3);
            *val = (vl >> (8 * k)) & 0xFFu;
            return ((base + (uint32_t)l) << 2) + k;
        }
    }
    return b;
}

__device__ __forceinline__ uint32_t f_range_max(const Win& W, const RawView& R, uint32_t a, uint32_t b) {
    const uint32_t ba = a >> 6, bl = (b - 1) >> 6;
    if (ba == bl) {
        if ((a & 63) == 0 && (b & 63) == 0) return W.m[ba];
        if (W.m[ba] == 0) return 0;
        return f_raw_max(W, R, a, b);
    }
    const uint32_t fb = (a + 63) >> 6, lb = b >> 6;
    uint32_t M = fb < lb ? f_sum_max(W, fb, lb) : 0;
    if ((a & 63) && W.m[ba] > M) {
        const uint32_t h = f_raw_max(W, R, a, (ba + 1) << 6);
        if (h > M) M = h;
    }
    if ((b & 63) && W.m[bl] > M) {
        const uint32_t t = f_raw_max(W, R, bl << 6, b);
        if (t > M) M = t;
    }
    return M;
}

__device__ __forceinline__ uint32_t f_first_geq(const Win& W, const RawView& R, uint32_t from, uint32_t to, uint32_t M,
                                                uint32_t* val) {
    uint32_t b = from >> 6;
    const uint32_t bend = (to - 1) >> 6;
    if ((from & 63) != 0 || b == bend) {
        const uint32_t bhi = (b + 1) << 6;
        const uint32_t bm = W.m[b];
        if (bm >= M) {
            const uint32_t a = (b << 6) + W.a[b];
            if (bm == M && a >= from) {
                if (a < to) { *val = M; return a; }
                return to;
            }
            const uint32_t e = min(bhi, to);
            const uint32_t r = f_raw_first_geq(W, R, from, e, M, val);
            if (r < e) return r;
        }
        if (b == bend) return to;
        b++;
    }
    while (b <= bend) {
        const uint32_t bh = f_sum_first_geq(W, b, bend + 1, M);
        if (bh > bend) return to;
        const uint32_t blo = bh << 6;
        const uint32_t bm = W.m[bh];
        const uint32_t a = blo + W.a[bh];
        if (bm == M) {
            if (a < to) { *val = M; return a; }
            return to;
        }
        const uint32_t e = min(blo + 64, to);
        const uint32_t r = f_raw_first_geq(W, R, blo, e, M, val);
        if (r < e) return r;
        if (e == to) return to;
        b = bh + 1;
    }
    return to;
}

// RAM step from window offset s; fhr = end of the file as a window offset
// (clamped: it is exact whenever it is within reach of the step)
__device__ __forceinline__ uint32_t f_next_ram(const Win& W, const RawView& R, const Prm& P, uint32_t fhr, uint32_t s) {
    if (fhr - s <= P.w) return fhr;
    const uint32_t limit = min(fhr, s + P.mx);
    const uint32_t t = s + P.w;
    const uint32_t M = f_range_max(W, R, s, t);
    const uint32_t j0 = max(t, s + P.mn - 1);
    if (j0 >= limit) return limit;
    if (M == 0) return j0 + 1;
    uint32_t val;
    const uint32_t j = f_first_geq(W, R, j0, limit, M, &val);
    return j < limit ? j + 1 : limit;
}

__device__ __forceinline__ uint32_t f_next_ae(const Win& W, const RawView& R, const Prm& P, uint32_t fhr, uint32_t s) {
    const uint32_t limit = min(fhr, s + P.mx);
    if (s + 1 >= limit) return limit;
    uint32_t p, v;
    {
        const uint32_t b = s >> 6;
        const uint32_t a = (b << 6) + W.a[b];
        if (a >= s && a < limit) {
            p = a;
            v = W.m[b];
        } else {
            const uint32_t e = min((b + 1) << 6, limit);
            v = f_raw_max(W, R, s, e);
            uint32_t val;
            p = v ? f_raw_first_geq(W, R, s, e, v, &val) : s;
        }
    }
    uint32_t cur = p + 1;
    for (;;) {
        const uint32_t t = max(p + P.w, s + P.mn - 1);
        if (t >= limit) return limit;
        if (v == 255) return t + 1;
        const uint32_t to = t + 1;
        if (cur & 63) {
            const uint32_t bc = cur >> 6, bhi = (bc + 1) << 6;
            const uint32_t bm = W.m[bc];
            if (bm > v) {
                const uint32_t a = (bc << 6) + W.a[bc];
                if (a >= cur && bhi <= to) {
                    p = a; v = bm; cur = a + 1;
                    continue;
                }
                const uint32_t e = min(bhi, to);
                uint32_t val;
                const uint32_t q = f_raw_first_geq(W, R, cur, e, v + 1, &val);
                if (q < e) {
                    p = q; v = val; cur = q + 1;
                    continue;
                }
            }
            if (bhi >= to) return to;
            cur = bhi;
        }
        const uint32_t bf = cur >> 6, bl = (to - 1) >> 6;
        const uint32_t bh = f_sum_first_geq(W, bf, bl + 1, v + 1);
        if (bh > bl) return to;
        const uint32_t blo = bh << 6;
        if (blo + 64 <= to) {
            p = blo + W.a[bh]; v = W.m[bh]; cur = p + 1;
            continue;
        }
        uint32_t val;
        const uint32_t q = f_raw_first_geq(W, R, blo, to, v + 1, &val);
        if (q < to) {
            p = q; v = val; cur = q + 1;
            continue;
        }
        return to;
    }
}

// MAXP step: the first target c with cmin <= c < cend ends the chunk after c.
// As window offsets: flw = flo + w (0 if before the window), fhr = fhi
// (clamped at 2^31), fhw = fhi - w (0 if the file has no room for a target
// or fhi - w is before the window).
__device__ __forceinline__ uint32_t f_next_maxp(const Win& W, const Prm& P, uint32_t flw, uint32_t fhr, uint32_t fhw,
                                                uint32_t s) {
    const uint32_t limit = min(fhr, s + P.mx);
    const uint32_t cmin = max(s + P.mn - 1, flw);
    const uint32_t cend = min(limit, fhw);
    if (cmin >= cend) return limit;
    const uint32_t b0 = cmin >> 6, b1 = ((cend - 1) >> 6) + 1, we = (b1 + 3) >> 2;
    for (uint32_t base = b0 >> 2; base < we; base += 32) {
        const uint32_t wi = base + lane_id();
        uint32_t c = 0xFFFFFFFFu;
        if (wi < we) {
            const uint32_t v = f_m4(W, wi);
            if (v != 0xFFFFFFFFu) {
#pragma unroll
                for (int k = 3; k >= 0; k--) {  // keep the smallest valid target of the word
                    const uint32_t bb = (wi << 2) + (uint32_t)k;
                    const uint32_t o = (v >> (8 * k)) & 0xFFu;
                    if (o == 0xFFu || bb < b0 || bb >= b1) continue;
                    const uint32_t cc = (bb << 6) + o;
                    if (cc >= cmin && cc < cend) c = cc;
                }
            }
        }
        const uint32_t bal = __ballot_sync(FULL, c != 0xFFFFFFFFu);
        if (bal) return __shfl_sync(FULL, c, __ffs((int)bal) - 1) + 1;
    }
    return limit;
}

// One or more chain steps from s, as w_advance(); the window path when the
// step stays inside W (every position it may touch is below s + max).
template <int RULE>
__device__ __forceinline__ uint64_t f_advance(const Win& W, const SumView& S, const RawView& R, const Prm& P,
                                              uint64_t flo, uint64_t fhi, uint64_t s, uint64_t stop, uint32_t* k,
                                              uint64_t* d) {
    // word reads may run 3 blocks past the last block a step needs
    if ((RULE == RULE_RAM || RULE == RULE_AE || RULE == RULE_MAXP) && s >= W.p0 &&
        s - W.p0 + (uint64_t)P.mx + 512 <= W.nb) {
        const uint32_t sr = (uint32_t)(s - W.p0);
        const uint32_t fhr = (uint32_t)umin64(fhi - W.p0, 0x80000000ull);  // fhi > s >= p0
        if (RULE == RULE_RAM || RULE == RULE_AE) {
            const uint32_t w = P.w;
            // the quiet-stretch test of w_advance: let it take such steps
            if (P.mn <= w + 1 && s + w < fhi && W.m[sr >> 6] == 0 && W.m[(sr + w - 1) >> 6] == 0)
                return w_advance<RULE>(S, R, P, flo, fhi, s, stop, k, d);
            const uint32_t e = RULE == RULE_RAM ? f_next_ram(W, R, P, fhr, sr) : f_next_ae(W, R, P, fhr, sr);
            *k = 1;
            *d = e - sr;
            return W.p0 + e;
        }
        if (RULE == RULE_MAXP) {
            const uint64_t flw64 = flo + P.w, fhw64 = fhi - P.w;
            const uint32_t flw = flw64 > W.p0 ? (uint32_t)umin64(flw64 - W.p0, 0x80000000ull) : 0u;
            const uint32_t fhw =
                (fhi > flw64 && fhw64 > W.p0) ? (uint32_t)umin64(fhw64 - W.p0, 0x80000000ull) : 0u;
            const uint64_t e1 = W.p0 + f_next_maxp(W, P, flw, fhr, fhw, sr);
            if (e1 == s + P.mx && e1 < fhi) return w_advance<RULE>(S, R, P, flo, fhi, s, stop, k, d);
            *k = 1;
            *d = e1 - s;
            return e1;
        }
    }
    return w_advance<RULE>(S, R, P, flo, fhi, s, stop, k, d);
}

}  // namespace cdc
