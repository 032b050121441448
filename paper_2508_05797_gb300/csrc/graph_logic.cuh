// graph_logic.cuh -- per-thread rules of the candidate-graph chain stage.
//
// Every chunk end that a chain can reach by a natural cut is a position y
// whose bytes satisfy a test that does not depend on the chunk's start
// (Section 2.1, the RAM and AE paragraphs; Section 3.3's compositions):
//
//   RAM  (min <= w + 1): the cut lands right after the first byte j >= s + w
//        with B[j] >= max B[s .. s+w); every byte between s + w and j is
//        below that maximum, so B[j] >= max B[j-w .. j). The candidate is
//        y = j + 1.
//   AE   (min <= w + 1): the cut lands w + 1 bytes after a target p with no
//        greater byte in (p, p+w], so B[p] >= max B[p+1 .. p+w]. The
//        candidate is y = p + w + 1.
//   MAXP: the cut lands right after a target c (strictly greater than every
//        byte within distance w, both windows inside the data): y = c + 1.
//
// A zero byte j (RAM) or p (AE) has an all-zero window; such "quiet"
// positions are left out (their chains are crossed in one step by
// advance()), so a candidate needs B[j] > 0 / B[p] > 0. The chain start
// (the first byte of the data) is a candidate of its own.
//
// F(y), the first candidate after y on the chain that starts at y, is one or
// a few next() steps (forced cuts at s + max and quiet stretches are not
// candidates). The chain of the whole input is then a path in the graph
// y -> F(y) that starts at the data's first byte; the kernels in graph.cu
// evaluate F for every candidate in parallel and resolve that path.
//
// Every function is __host__ __device__ so that the host tests can run the
// same code against the CPU oracle.
#pragma once
#include <stdint.h>

#include "chain_logic.cuh"

namespace cdc {

// source byte of candidate y = y - shift: j (RAM), p (AE) or c (MAXP)
template <int RULE>
CDC_HD uint64_t cand_shift(const Prm& P) {
    return RULE == RULE_AE ? (uint64_t)P.w + 1 : 1;
}

// Source positions that can make a candidate in [lo, hi): [*a, *b).
template <int RULE>
CDC_HD void cand_source_range(const Prm& P, uint64_t lo, uint64_t hi, uint64_t* a, uint64_t* b) {
    const uint64_t w = P.w;
    uint64_t s0, s1;
    if (RULE == RULE_RAM) {
        s0 = lo + w;                       // the window [j - w, j) inside the data
        s1 = hi >= 1 ? hi - 1 : 0;         // y = j + 1 < hi (y = hi ends the data)
    } else if (RULE == RULE_AE) {
        s0 = lo;
        s1 = hi >= w + 1 ? hi - w - 1 : 0;  // y = p + w + 1 < hi
    } else {
        s0 = lo + w;                        // both windows inside the data
        s1 = hi >= w ? hi - w : 0;
    }
    *a = s0;
    *b = s1 > s0 ? s1 : s0;
}

// Is the byte at source position q (inside the source range) a candidate?
template <int RULE>
CDC_HD bool cand_at(const SumView& S, const RawView& R, const Prm& P, uint64_t q) {
    if (RULE == RULE_MAXP) return S.m(q >> 6) == (uint32_t)(q & 63);
    const uint32_t x = R.byte(q);
    if (x == 0) return false;
    if (x == 255) return true;
    if (RULE == RULE_RAM) return range_max(S, R, q - P.w, q) <= x;
    return range_max(S, R, q + 1, q + P.w + 1) <= x;
}

// Is position y a candidate of the data [lo, hi)?
template <int RULE>
CDC_HD bool is_cand(const SumView& S, const RawView& R, const Prm& P, uint64_t lo, uint64_t hi, uint64_t y) {
    uint64_t a, b;
    cand_source_range<RULE>(P, lo, hi, &a, &b);
    const uint64_t sh = cand_shift<RULE>(P);
    if (y < sh) return false;
    const uint64_t q = y - sh;
    if (q < a || q >= b) return false;
    return cand_at<RULE>(S, R, P, q);
}

// Candidates among the source bytes of block b that lie in [qa, qb): bit o
// of the result is set when source position 64 b + o makes a candidate.
// Summaries first: a block whose maximum is below the maximum of the whole
// blocks that every one of its bytes' windows covers has none (for RAM on
// random bytes that rejects about four blocks in five); the others are read
// once and each byte is tested against its window exactly.
template <int RULE>
CDC_HD uint64_t block_cands(const SumView& S, const RawView& R, const Prm& P, uint64_t b, uint64_t qa,
                            uint64_t qb) {
    const uint64_t b0 = b << 6;
    const uint64_t oa = qa > b0 ? qa - b0 : 0, ob = qb < b0 + 64 ? qb - b0 : 64;
    if (oa >= ob) return 0;
    if (RULE == RULE_MAXP) {
        const uint32_t o = S.m(b);
        return (o != 0xFFu && o >= oa && o < ob) ? (1ull << o) : 0;
    }
    const uint32_t bm = S.m(b);
    if (bm == 0) return 0;
    const uint64_t w = P.w;
    // whole blocks inside the window of every byte of block b: [fb, fe)
    uint64_t fb, fe;
    if (RULE == RULE_RAM) {
        fb = (b0 + 63 + 63 >= w) ? (b0 + 126 - w) >> 6 : 0;  // window [q - w, q)
        fe = b;
    } else {
        fb = b + 1;  // window [q + 1, q + w + 1)
        fe = (b0 + w + 1) >> 6;
    }
    const uint32_t L = fb < fe ? sum_max(S, fb, fe) : 0;
    if (bm < L) return 0;
    // (w >= 64: a block holding a source byte lies inside the data, from its
    // first byte for RAM, up to its last byte for AE)
    uint32_t wd[16];
    uint64_t mask = 0;
    if (RULE == RULE_RAM) {
        R.block(b0, b0 + ob, wd);
        uint32_t pm = 0;  // maximum of the block's bytes before the current one
        for (uint32_t o = 0; o < ob; o++) {
            const uint32_t x = (wd[o >> 2] >> (8 * (o & 3))) & 0xFFu;
            if (o >= oa && x != 0 && x >= L && x >= pm) {
                bool ok = true;
                if (x != 255) {
                    const uint64_t q = b0 + o;
                    const uint64_t h1 = fb << 6;  // bytes [q - w, h1) lie before the whole blocks
                    if (q - w < h1 && range_max(S, R, q - w, h1) > x) ok = false;
                }
                if (ok) mask |= 1ull << o;
            }
            if (x > pm) pm = x;
        }
    } else {
        R.block(b0 + oa, b0 + 64, wd);
        uint32_t sm = 0;  // maximum of the block's bytes after the current one
        for (int oi = 63; oi >= (int)oa; oi--) {
            const uint32_t o = (uint32_t)oi;
            const uint32_t x = (wd[o >> 2] >> (8 * (o & 3))) & 0xFFu;
            if (o < ob && x != 0 && x >= L && x >= sm) {
                bool ok = true;
                if (x != 255) {
                    const uint64_t q = b0 + o;
                    const uint64_t t0 = fe > b + 1 ? fe << 6 : b0 + 64;  // bytes [t0, q + w + 1) remain
                    if (t0 < q + w + 1 && range_max(S, R, t0, q + w + 1) > x) ok = false;
                }
                if (ok) mask |= 1ull << o;
            }
            if (x > sm) sm = x;
        }
    }
    return mask;
}

// ---- scans that skip 4 KiB superblocks by their summaries ----------------------
//
// The chain steps of chain_logic.cuh scan block summaries one 16-block group
// after another. A candidate's F walk can cross zero runs and target-less
// stretches of hundreds of kilobytes, so the walks here first skip whole
// superblocks (64 blocks), 16 superblock summaries (64 KiB) per 16-byte load.

// first superblock in [q0, q1) whose summary is >= M (1 <= M <= 255); q1 if none
CDC_HD uint64_t sup_first_geq(const uint8_t* sup, uint64_t q0, uint64_t q1, uint32_t M) {
    const uint32_t K = ge_key(M);
    for (uint64_t g = q0 >> 4, ge = (q1 + 15) >> 4; g < ge; g++) {
        uint32_t w[4];
#if defined(__CUDA_ARCH__)
        const uint4 v = *reinterpret_cast<const uint4*>(sup + (g << 4));
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
#else
        for (int k = 0; k < 4; k++) w[k] = reinterpret_cast<const uint32_t*>(sup + (g << 4))[k];
#endif
        CDC_UNROLL
        for (int k = 0; k < 4; k++) {
            const uint64_t wi = 4 * g + (uint64_t)k;
            const uint32_t f = ge_flags(clip_word(w[k], wi, q0, q1), K);
            if (f) return (wi << 2) + (uint32_t)((ffs32(f) - 1) >> 3);
        }
    }
    return q1;
}

// first block in [b0, b1) with m[] >= M (M >= 1), skipping superblocks whose
// summary is below M (RAM / AE summaries: the superblock maximum); b1 if none
CDC_HD uint64_t sum_first_geq_far(const SumView& S, uint64_t b0, uint64_t b1, uint32_t M) {
    uint64_t b = b0;
    while (b < b1) {
        if ((b & 63) || !S.sup || b + 64 > b1) {
            // up to the next superblock boundary (or the end) block by block
            const uint64_t e = umin64(b1, (b + 64) & ~63ull);
            const uint64_t h = sum_first_geq(S, b, e, M);
            if (h < e) return h;
            b = e;
            continue;
        }
        const uint64_t q = sup_first_geq(S.sup, b >> 6, b1 >> 6, M);  // whole superblocks only
        if (q >= (b1 >> 6)) {
            b = (b1 >> 6) << 6;  // the partial superblock at the end, if any
            continue;
        }
        const uint64_t e = (q + 1) << 6;
        const uint64_t h = sum_first_geq(S, q << 6, e, M);
        if (h < e) return h;
        b = e;  // (cannot happen: the superblock holds a block >= M)
    }
    return b1;
}

// Range Scan (GEQ) as first_geq(), with the superblock skips
CDC_HD uint64_t first_geq_far(const SumView& S, const RawView& R, uint64_t from, uint64_t to, uint32_t M,
                              uint32_t* val) {
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
            const uint64_t r = raw_first_geq(R, from, e, M, val);
            if (r < e) return r;
        }
        if (b == bend) return to;
        b++;
    }
    while (b <= bend) {
        const uint64_t bh = sum_first_geq_far(S, b, bend + 1, M);
        if (bh > bend) return to;
        const uint64_t blo = bh << 6;
        const uint32_t bm = S.m(bh);
        const uint64_t a = blo + S.a(bh);
        if (bm == M) {
            if (a < to) { *val = M; return a; }
            return to;
        }
        const uint64_t e = umin64(blo + 64, to);
        const uint64_t r = raw_first_geq(R, blo, e, M, val);
        if (r < e) return r;
        if (e == to) return to;
        b = bh + 1;
    }
    return to;
}

// RAM next(s) with the long scan over superblocks (equals next_ram)
CDC_HD uint64_t next_ram_far(const SumView& S, const RawView& R, const Prm& P, uint64_t fhi, uint64_t s) {
    if (fhi - s <= P.w) return fhi;
    const uint64_t limit = umin64(fhi, s + P.mx);
    const uint64_t t = s + P.w;
    const uint32_t M = range_max(S, R, s, t);
    const uint64_t j0 = umax64(t, s + P.mn - 1);
    if (j0 >= limit) return limit;
    if (M == 0) return j0 + 1;
    uint32_t val;
    const uint64_t j = first_geq_far(S, R, j0, limit, M, &val);
    return j < limit ? j + 1 : limit;
}

// first MAXP target c with c0 <= c < c1 (per-block target offsets, per-
// superblock target counts), skipping superblocks without one; c1 if none
CDC_HD uint64_t first_target_far(const SumView& S, uint64_t c0, uint64_t c1) {
    uint64_t p = c0;
    while (p < c1) {
        if ((p & 4095) == 0 && S.sup && p + 4096 <= c1) {
            const uint64_t q = sup_first_geq(S.sup, p >> 12, c1 >> 12, 1);
            if (q > (p >> 12)) {
                p = q << 12;
                continue;
            }
        }
        // blocks of p's superblock, 16 target bytes per load
        const uint64_t pe = umin64(c1, (p + 4096) & ~4095ull);
        for (uint64_t b = p >> 6, be = (pe + 63) >> 6; b < be;) {
            uint32_t w[4];
            S.m16(b >> 4, w);
            bool found = false;
            uint64_t c = 0;
            CDC_UNROLL
            for (int k = 0; k < 4; k++) {
                for (uint32_t j = 0; j < 4 && !found; j++) {
                    const uint64_t bb = ((b >> 4) << 4) + 4 * (uint64_t)k + j;
                    const uint32_t o = (w[k] >> (8 * j)) & 0xFFu;
                    if (bb < (p >> 6) || bb >= be || o == 0xFFu) continue;
                    const uint64_t cc = (bb << 6) + o;
                    if (cc >= p && cc < pe) {
                        c = cc;
                        found = true;
                    }
                }
            }
            if (found) return c;
            b = ((b >> 4) + 1) << 4;
        }
        p = pe;
    }
    return c1;
}

CDC_HD uint64_t next_maxp_far(const SumView& S, const Prm& P, uint64_t flo, uint64_t fhi, uint64_t s) {
    const uint64_t limit = umin64(fhi, s + P.mx);
    const uint64_t cmin = umax64(s + P.mn - 1, flo + P.w);
    const uint64_t cend = fhi > flo + P.w ? umin64(limit, fhi - P.w) : 0;
    if (cmin >= cend) return limit;
    const uint64_t c = first_target_far(S, cmin, cend);
    return c < cend ? c + 1 : limit;
}

// advance() with the superblock scans (the same steps)
template <int RULE>
CDC_HD uint64_t advance_far(const SumView& S, const RawView& R, const Prm& P, uint64_t flo, uint64_t fhi,
                            uint64_t s, uint64_t stop, uint32_t* k, uint64_t* d) {
    if (RULE == RULE_RAM || RULE == RULE_AE) {
        const uint64_t w = P.w, st = w + 1;
        if (P.mn <= st && s + w < fhi && S.m(s >> 6) == 0 && S.m((s + w - 1) >> 6) == 0) {
            const uint64_t kstop = (stop - 1 - s) / st + 1;
            const uint64_t kfhi = (fhi - 1 - s - w) / st + 1;
            const uint64_t kmax = kstop < kfhi ? kstop : kfhi;
            const uint64_t bound = s + (kmax - 1) * st + w + 1;
            uint32_t val;
            const uint64_t z = first_geq_far(S, R, s, bound, 1, &val);  // first non-zero byte
            const uint64_t kz = z > s + w ? (z - 1 - s - w) / st + 1 : 0;
            const uint64_t kk = kz < kmax ? kz : kmax;
            if (kk >= 2) {
                *k = (uint32_t)kk;
                *d = st;
                return s + kk * st;
            }
        }
        const uint64_t e = RULE == RULE_RAM ? next_ram_far(S, R, P, fhi, s) : next_ae(S, R, P, fhi, s);
        *k = 1;
        *d = e - s;
        return e;
    }
    const uint64_t e1 = next_maxp_far(S, P, flo, fhi, s);
    if (e1 == s + P.mx && e1 < fhi) {
        const uint64_t mx = P.mx;
        const uint64_t c0 = umax64(s + P.mn - 1, flo + P.w);
        const uint64_t cend = fhi > flo + P.w ? fhi - P.w : 0;
        const uint64_t kstop = (stop - 1 - s) / mx + 1;
        const uint64_t kfhi = (fhi - s) / mx;
        const uint64_t kmax = kstop < kfhi ? kstop : kfhi;
        if (kmax >= 2) {
            const uint64_t lim = umin64(cend, s + kmax * mx);
            const uint64_t c = c0 < lim ? first_target_far(S, c0, lim) : lim;
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

// ---- window maxima from running maxima inside superblocks ------------------
//
// pre[b] = max m[] over the blocks of b's 4 KiB superblock up to b, suf[b] =
// from b to the superblock's end (written by the summary kernel), sup[q] = the
// superblock's maximum. The maximum of whole blocks [fb, lb) spanning two or
// more superblocks is max(suf[fb], sup of the superblocks between, pre[lb - 1]),
// two or three reads for the windows of the configured workloads; a range
// inside one superblock that touches either end is one read.
struct PreSuf {
    const uint8_t* pre;  // null: no running maxima
    const uint8_t* suf;
};

// maximum of the whole blocks [fb, lb) (fb < lb)
CDC_HD uint32_t whole_max(const SumView& S, const PreSuf& V, uint64_t fb, uint64_t lb) {
    if (!V.pre || !S.sup) return sum_max(S, fb, lb);
    const uint64_t q0 = fb >> 6, q1 = (lb - 1) >> 6;
    if (q0 == q1) {
        if ((fb & 63) == 0) return V.pre[lb - 1];
        if ((lb & 63) == 0) return V.suf[fb];
        return sum_max(S, fb, lb);
    }
    uint32_t M = V.suf[fb];
    const uint32_t t = V.pre[lb - 1];
    if (t > M) M = t;
    for (uint64_t q = q0 + 1; q < q1 && M < 255; q++) {
        const uint32_t u = S.sup[q];
        if (u > M) M = u;
    }
    return M;
}

// Extreme Byte Search over [a, b) with the running maxima (equals range_max)
CDC_HD uint32_t range_max_t(const SumView& S, const PreSuf& V, const RawView& R, uint64_t a, uint64_t b) {
    const uint64_t ba = a >> 6, bl = (b - 1) >> 6;
    if (ba == bl) return range_max(S, R, a, b);
    const uint64_t fb = (a + 63) >> 6, lb = b >> 6;
    uint32_t M = fb < lb ? whole_max(S, V, fb, lb) : 0;
    if (M == 255) return 255;
    if ((a & 63) && S.m(ba) > M) {
        const uint32_t h = raw_max(R, a, (ba + 1) << 6);
        if (h > M) M = h;
    }
    if ((b & 63) && S.m(bl) > M) {
        const uint32_t t = raw_max(R, bl << 6, b);
        if (t > M) M = t;
    }
    return M;
}

// RAM next(s) (equals next_ram). *nat: the cut is natural (a byte >= the
// window maximum was found), then *val is that byte.
CDC_HD uint64_t next_ram_t(const SumView& S, const PreSuf& T, const RawView& R, const Prm& P, uint64_t fhi,
                           uint64_t s, bool* nat, uint32_t* val) {
    *nat = false;
    if (fhi - s <= P.w) return fhi;
    const uint64_t limit = umin64(fhi, s + P.mx);
    const uint64_t t = s + P.w;
    const uint64_t j0 = umax64(t, s + P.mn - 1);
    if (j0 >= limit) return limit;
    const uint32_t M = range_max_t(S, T, R, s, t);
    if (M == 0) {
        *nat = true;
        *val = R.byte(j0);
        return j0 + 1;
    }
    const uint64_t j = first_geq_far(S, R, j0, limit, M, val);
    if (j < limit) {
        *nat = true;
        return j + 1;
    }
    return limit;
}

// AE-Max next(s) over the (possibly complemented) bytes, w >= 64 (equals
// next_ae): before scanning a target's window for a greater byte, the table
// tells whether the window holds one at all. *nat: the cut ends a target's
// window, then *val is the target's byte.
CDC_HD uint64_t next_ae_t(const SumView& S, const PreSuf& T, const RawView& R, const Prm& P, uint64_t fhi,
                          uint64_t s, bool* nat, uint32_t* val) {
    *nat = false;
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
            raw_max_first(R, s, umin64((b + 1) << 6, limit), &v, &p);
        }
    }
    uint64_t cur = p + 1;
    for (;;) {
        const uint64_t t = umax64(p + P.w, s + P.mn - 1);
        if (t >= limit) return limit;
        if (v == 255) {
            *nat = true;
            *val = v;
            return t + 1;
        }
        const uint64_t to = t + 1;
        // the window [cur, to) holds no byte above v: the target ends the chunk
        if (cur < to && range_max_t(S, T, R, cur, to) <= v) {
            *nat = true;
            *val = v;
            return to;
        }
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
                uint32_t vv;
                const uint64_t q = raw_first_geq(R, cur, e, v + 1, &vv);
                if (q < e) {
                    p = q; v = vv; cur = q + 1;
                    continue;
                }
            }
            if (bhi >= to) {
                *nat = true;
                *val = v;
                return to;
            }
            cur = bhi;
        }
        const uint64_t bf = cur >> 6, bl = (to - 1) >> 6;
        const uint64_t bh = sum_first_geq(S, bf, bl + 1, v + 1);
        if (bh > bl) {
            *nat = true;
            *val = v;
            return to;
        }
        const uint64_t blo = bh << 6;
        if (blo + 64 <= to) {
            p = blo + S.a(bh); v = S.m(bh); cur = p + 1;
            continue;
        }
        uint32_t vv;
        const uint64_t q = raw_first_geq(R, blo, to, v + 1, &vv);
        if (q < to) {
            p = q; v = vv; cur = q + 1;
            continue;
        }
        *nat = true;
        *val = v;
        return to;
    }
}

// F(y): from the chunk start y (a candidate or the data's first byte), take
// chain steps until the chain reaches a candidate or the end of the data.
// Returns that position (hi for the end) and sets *n to the number of chunk
// ends on the way (the returned position included, >= 1). A natural cut is a
// candidate exactly when its byte (RAM) or its target's byte (AE) is not zero
// (the scan that found it already compared it with the whole window); only
// forced cuts and the end of a quiet run take the full test.
template <int RULE>
CDC_HD uint64_t cand_next_t(const SumView& S, const PreSuf& T, const RawView& R, const Prm& P, uint64_t lo,
                            uint64_t hi, uint64_t y, uint32_t* n) {
    uint64_t s = y;
    uint32_t c = 0;
    for (;;) {
        if (RULE == RULE_RAM || RULE == RULE_AE) {
            const uint64_t w = P.w, st = w + 1;
            if (P.mn <= st && s + w < hi && S.m(s >> 6) == 0 && S.m((s + w - 1) >> 6) == 0) {
                // a zero run: cuts every w + 1 bytes (advance_far's quiet steps);
                // their cut bytes are zero, so none of them is a candidate
                const uint64_t kmax = (hi - 1 - s - w) / st + 1;
                const uint64_t bound = s + (kmax - 1) * st + w + 1;
                uint32_t val;
                const uint64_t z = first_geq_far(S, R, s, bound, 1, &val);
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
            bool nat;
            uint32_t val;
            const uint64_t e = RULE == RULE_RAM ? next_ram_t(S, T, R, P, hi, s, &nat, &val)
                                                : next_ae_t(S, T, R, P, hi, s, &nat, &val);
            c++;
            if (e >= hi) {
                *n = c;
                return hi;
            }
            if (nat ? val != 0 : is_cand<RULE>(S, R, P, lo, hi, e)) {
                *n = c;
                return e;
            }
            s = e;
        } else {
            uint32_t k;
            uint64_t d;
            const uint64_t e = advance_far<RULE>(S, R, P, lo, hi, s, hi, &k, &d);
            c += k;
            if (e >= hi) {
                *n = c;
                return hi;
            }
            if (is_cand<RULE>(S, R, P, lo, hi, e)) {
                *n = c;
                return e;
            }
            s = e;
        }
    }
}

template <int RULE>
CDC_HD uint64_t cand_next(const SumView& S, const RawView& R, const Prm& P, uint64_t lo, uint64_t hi, uint64_t y,
                          uint32_t* n) {
    const PreSuf T{nullptr, nullptr};
    return cand_next_t<RULE>(S, T, R, P, lo, hi, y, n);
}

// ---- F from the sorted candidate list ---------------------------------------
//
// A natural cut lands on a candidate, so most of F needs no scan of the bytes:
//   RAM : the cut byte is the first byte >= M (the window maximum) at or past
//         s + w; that byte is itself a candidate, and every candidate before
//         it in that range is below M -- the first listed candidate from
//         s + w whose byte is >= M. With none before s + max the chunk is
//         forced to end at s + max: F is that position if it is listed, else
//         the list decides the next chunk from there the same way.
//   AE  : the cut follows the first target (a strict prefix maximum from s)
//         with no greater byte in its window -- the first listed candidate q
//         >= s whose byte exceeds every byte of [s, q).
//   MAXP: the first listed target at or past max(s + min - 1, lo + w).
// The list holds the candidates at positions base + pos[i] (increasing), with
// their source bytes val[i], and is complete for positions below `cover`.

constexpr uint32_t LIST_GENERIC = 0xFFFFFFFFu;  // the list cannot decide: step the chain

struct CandList {
    const uint32_t* pos;
    const uint8_t* val;
    uint32_t n;
    uint64_t base, cover;
    const uint8_t* gmax;  // maximum of val[32 g .. 32 g + 31] per group g, or null
};

// first index >= k whose position is <= ymax and whose byte is >= M; L.n if none
CDC_HD uint32_t list_first_geq(const CandList& L, uint32_t k, uint64_t ymax, uint32_t M) {
    while (k < L.n) {
        if (L.gmax && (k & 31) == 0 && L.gmax[k >> 5] < M) {
            // the whole group is below M: skip it unless it reaches past ymax
            const uint32_t last = k + 31 < L.n ? k + 31 : L.n - 1;
            if (L.base + L.pos[last] > ymax) return L.n;
            k += 32;
            continue;
        }
        if (L.base + L.pos[k] > ymax) return L.n;
        if (L.val[k] >= M) return k;
        k++;
    }
    return L.n;
}

CDC_HD uint32_t list_lower_bound(const CandList& L, uint64_t y) {
    if (y <= L.base) return 0;
    const uint64_t r = y - L.base;
    uint32_t lo = 0, hi = L.n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint64_t)L.pos[mid] < r) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Index in L of F(s) when the list decides the chain from s (natural cuts, and
// for RAM forced cuts before one), else LIST_GENERIC; *cnt = the chunk ends up
// to F. wmax(a, b) is the maximum byte of [a, b) (a < b); R reads single
// bytes (AE's start byte).
template <int RULE, class WMax>
CDC_HD uint32_t list_next(const CandList& L, const WMax& wmax, const RawView& R, const Prm& P, uint64_t lo,
                          uint64_t hi, uint64_t s, uint32_t* cnt) {
    const uint64_t w = P.w;
    const uint64_t limit = umin64(hi, s + P.mx);
    *cnt = 1;
    if (RULE == RULE_RAM) {
        uint64_t s0 = s;
        for (uint32_t c = 1; c <= 4; c++) {
            const uint64_t lim = umin64(hi, s0 + P.mx);
            if (hi - s0 <= w) return LIST_GENERIC;
            const uint64_t j0 = s0 + w;  // min <= w + 1
            if (j0 >= lim) return LIST_GENERIC;
            const uint32_t M = wmax(s0, j0);
            if (M == 0) return LIST_GENERIC;
            const uint64_t ymax = umin64(lim, L.cover);
            const uint32_t k = list_first_geq(L, list_lower_bound(L, j0 + 1), ymax, M);
            if (k < L.n) {
                *cnt = c;
                return k;
            }
            // no natural cut up to ymax: a forced cut at lim, if the list covers it
            if (lim > L.cover || lim >= hi) return LIST_GENERIC;
            const uint32_t kf = list_lower_bound(L, lim);
            if (kf < L.n && L.base + L.pos[kf] == lim) {
                *cnt = c;
                return kf;
            }
            s0 = lim;
        }
        return LIST_GENERIC;
    }
    if (RULE == RULE_AE) {
        if (s + 1 >= limit || s + w >= limit) return LIST_GENERIC;
        const uint32_t vs = R.byte(s);
        if (vs == 0 && wmax(s + 1, s + w + 1) == 0) return LIST_GENERIC;  // a quiet cut at s + w + 1
        int mr = -1;  // maximum of [s, q)
        uint64_t qp = s;
        for (uint32_t k = list_lower_bound(L, s + w + 1); k < L.n; k++) {
            const uint64_t y = L.base + L.pos[k];
            if (y > L.cover) return LIST_GENERIC;
            const uint64_t q = y - w - 1;
            if (q + w >= limit) return LIST_GENERIC;
            if (q > qp) {
                const int m = (int)wmax(qp, q);
                if (m > mr) mr = m;
            }
            if ((int)L.val[k] > mr) return k;
            qp = q;
        }
        return LIST_GENERIC;
    }
    const uint64_t cmin = umax64(s + P.mn - 1, lo + w);
    const uint64_t cend = hi > lo + w ? umin64(limit, hi - w) : 0;
    if (cmin >= cend) return LIST_GENERIC;
    const uint32_t k = list_lower_bound(L, cmin + 1);
    if (k >= L.n) return LIST_GENERIC;
    const uint64_t y = L.base + L.pos[k];
    if (y > L.cover) return LIST_GENERIC;
    return y - 1 < cend ? k : LIST_GENERIC;
}

// window maximum over the block summaries (and running maxima, if any)
struct WMaxSum {
    const SumView* S;
    const PreSuf* T;
    const RawView* R;
    CDC_HD uint32_t operator()(uint64_t a, uint64_t b) const { return range_max_t(*S, *T, *R, a, b); }
};

}  // namespace cdc
