// chain_logic.cuh -- per-thread chunk rules over block summaries (RAM, AE, MAXP).
//
// next(s) returns the end of the chunk that starts at s, exactly as the
// sequential rules of arxiv 2508.05797 define it (Section 2.1, Section 3.3;
// the min / max rule of Section 2.1). What makes it fast is where it looks:
// instead of every byte it reads per-64-byte-block summaries written by the
// summary kernel, and touches raw bytes only where a summary cannot decide.
//
//   * Extreme Byte Search (Section 3.1) over a window becomes a max over the
//     block maxima of the whole blocks inside it (4 blocks per 32-bit word,
//     combined with byte-wise SIMD max), plus raw reads of the partial end
//     blocks only when their block maximum could raise the result.
//   * Range Scan (Section 3.2) for the first byte >= M becomes a packed
//     compare over the block maxima (4 per word); in the hit block the first
//     occurrence of the block maximum is the answer when that maximum equals
//     M, otherwise the block's bytes are scanned.
//   * AE walks its targets block by block: inside a block every target but
//     the last has its next greater byte within 63 bytes, so with w >= 64
//     none of them can end a chunk, and the walk jumps to the block's first
//     maximum.
//   * MAXP reads the target found by the summary kernel in each block (at
//     most one per block when w >= 63) and keeps the first one that fits
//     the chunk-size rules.
//
// Positions are byte offsets from a 64-byte aligned base ("physical"); a
// file occupies [flo, fhi). Every function is __host__ __device__ so that the
// same code can be checked on the CPU.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define CDC_HD __host__ __device__ __forceinline__
#define CDC_UNROLL _Pragma("unroll")
#else
#define CDC_HD inline
#define CDC_UNROLL
#endif

namespace cdc {

constexpr uint32_t NONE_SLOT = 0xFFu;

CDC_HD uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
CDC_HD uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// ---- byte-wise SIMD helpers (device intrinsics; portable fallbacks on the host)
CDC_HD uint32_t vmax4(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __vmaxu4(a, b);
#else
    uint32_t r = 0;
    for (int k = 0; k < 4; k++) {
        uint32_t x = (a >> (8 * k)) & 0xFFu, y = (b >> (8 * k)) & 0xFFu;
        r |= (x > y ? x : y) << (8 * k);
    }
    return r;
#endif
}

// 0xFF in each byte where a >= b (unsigned)
CDC_HD uint32_t vcmpge4(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __vcmpgeu4(a, b);
#else
    uint32_t r = 0;
    for (int k = 0; k < 4; k++)
        if (((a >> (8 * k)) & 0xFFu) >= ((b >> (8 * k)) & 0xFFu)) r |= 0xFFu << (8 * k);
    return r;
#endif
}

CDC_HD uint32_t vcmpeq4(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __vcmpeq4(a, b);
#else
    uint32_t r = 0;
    for (int k = 0; k < 4; k++)
        if (((a >> (8 * k)) & 0xFFu) == ((b >> (8 * k)) & 0xFFu)) r |= 0xFFu << (8 * k);
    return r;
#endif
}

CDC_HD int ffs32(uint32_t x) {
#if defined(__CUDA_ARCH__)
    return __ffs((int)x);
#else
    return __builtin_ffs((int)x);
#endif
}

// largest byte of a word
CDC_HD uint32_t hmax4(uint32_t v) {
    v = vmax4(v, v >> 16);
    v = vmax4(v, v >> 8);
    return v & 0xFFu;
}

// ---- bytes in 16-bit lanes: a word's bytes 0 and 2 ("even") and 1 and 3
// ("odd") each go into the low half of a 16-bit lane, where native 16x2
// integer operations handle two bytes at a time.
CDC_HD uint32_t vmax2(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __vmaxu2(a, b);
#else
    uint32_t lo = (a & 0xFFFFu) > (b & 0xFFFFu) ? (a & 0xFFFFu) : (b & 0xFFFFu);
    uint32_t hi = (a >> 16) > (b >> 16) ? (a >> 16) : (b >> 16);
    return lo | (hi << 16);
#endif
}

// running maximum of the bytes of the words added
struct ByteMax {
    uint32_t e = 0, o = 0;
    CDC_HD void add(uint32_t x) {
        e = vmax2(e, x & 0x00FF00FFu);
        o = vmax2(o, (x >> 8) & 0x00FF00FFu);
    }
    CDC_HD uint32_t get() const {
        const uint32_t m = vmax2(e, o);
        return (m & 0xFFFFu) > (m >> 16) ? (m & 0xFFFFu) : (m >> 16);
    }
    // some byte is 255: the maximum cannot grow
    CDC_HD bool full() const { return ((vmax2(e, o) + 0x00010001u) & 0x01000100u) != 0; }
};

// Lane offset K for ge_flags(): (0x8000 - M) in both 16-bit lanes, 1 <= M <= 255.
CDC_HD uint32_t ge_key(uint32_t M) { return (0x8000u - M) * 0x00010001u; }

// Bit 7 of byte k is set where byte k of x is >= M (K = ge_key(M)): a byte
// plus 0x8000 - M reaches bit 15 of its lane exactly when it is >= M, and no
// lane overflows into the next.
CDC_HD uint32_t ge_flags(uint32_t x, uint32_t K) {
    const uint32_t e = (x & 0x00FF00FFu) + K, o = ((x >> 8) & 0x00FF00FFu) + K;
    return ((e >> 8) & 0x00800080u) | (o & 0x80008000u);
}

// keep the bytes of word i of a block (block bytes [4i, 4i+4)) whose block
// offsets lie in [oa, ob); 0 <= oa < ob <= 64
CDC_HD uint32_t clip_in_block(uint32_t v, uint32_t i, uint32_t oa, uint32_t ob) {
    const uint32_t lo = 4 * i;
    if (lo + 4 <= oa || lo >= ob) return 0;
    if (lo < oa) v &= 0xFFFFFFFFu << (8 * (oa - lo));
    if (lo + 4 > ob) v &= 0xFFFFFFFFu >> (8 * (lo + 4 - ob));
    return v;
}

// keep the bytes of word `wi` (bytes [4wi, 4wi+4)) that lie in [a, b)
CDC_HD uint32_t clip_word(uint32_t v, uint64_t wi, uint64_t a, uint64_t b) {
    uint64_t lo = wi << 2;
    if (lo + 4 <= a || lo >= b) return 0;  // no byte of the word in [a, b)
    if (lo < a) v &= 0xFFFFFFFFu << (8 * (uint32_t)(a - lo));
    if (lo + 4 > b) v &= 0xFFFFFFFFu >> (8 * (uint32_t)(lo + 4 - b));
    return v;
}

// ---- data views ------------------------------------------------------------

// Raw bytes of the input. `inv` = 0xFFFFFFFF reads 255 - b (AE-Min runs the
// AE-Max rules on complemented bytes). Callers only read words holding at
// least one byte of [flo, fhi), which lie inside the buffer's 16-byte granules.
struct RawView {
    const uint8_t* base;
    uint32_t inv;
    CDC_HD uint32_t word(uint64_t wi) const {
#if defined(__CUDA_ARCH__)
        return __ldg(reinterpret_cast<const uint32_t*>(base) + wi) ^ inv;
#else
        return reinterpret_cast<const uint32_t*>(base)[wi] ^ inv;
#endif
    }
    CDC_HD uint32_t byte(uint64_t p) const { return (word(p >> 2) >> (8 * (uint32_t)(p & 3))) & 0xFFu; }
    // the 16-byte granule gi as 4 words
    CDC_HD void granule(uint64_t gi, uint32_t w[4]) const {
#if defined(__CUDA_ARCH__)
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(base) + gi);
        w[0] = v.x ^ inv; w[1] = v.y ^ inv; w[2] = v.z ^ inv; w[3] = v.w ^ inv;
#else
        const uint32_t* p = reinterpret_cast<const uint32_t*>(base) + 4 * gi;
        for (int k = 0; k < 4; k++) w[k] = p[k] ^ inv;
#endif
    }
    // Words of the block holding [a, b) (a < b <= end of that 64-byte block):
    // the granules that meet [a, b) are loaded (all at once), the others read 0.
    CDC_HD void block(uint64_t a, uint64_t b, uint32_t w[16]) const {
        const uint64_t g0 = a >> 4, g1 = (b - 1) >> 4, gb = (a >> 6) << 2;
        CDC_UNROLL
        for (int k = 0; k < 4; k++) {
            const uint64_t g = gb + (uint64_t)k;
            if (g >= g0 && g <= g1) {
                granule(g, w + 4 * k);
            } else {
                w[4 * k] = w[4 * k + 1] = w[4 * k + 2] = w[4 * k + 3] = 0;
            }
        }
    }
};

// Per-block summaries: m[b] (block maximum, or for MAXP the offset of the
// block's target / 0xFF) and a[b] (offset of the first maximum). A window of
// blocks [wb0, wb0 + wn) may be staged in fast memory (sm, sa); other blocks
// are read from the global arrays (gm, ga). wb0 is a multiple of 16.
struct SumView {
    const uint8_t* gm;
    const uint8_t* ga;
    const uint8_t* sm;
    const uint8_t* sa;
    uint64_t wb0, wn;
    const uint8_t* sup;  // per 4 KiB superblock: max byte (RAM/AE) or target count (MAXP); may be null
    CDC_HD uint32_t m(uint64_t b) const {
        uint64_t r = b - wb0;
        return (b >= wb0 && r < wn) ? sm[r] : gm[b];
    }
    CDC_HD uint32_t a(uint64_t b) const {
        uint64_t r = b - wb0;
        return (b >= wb0 && r < wn) ? sa[r] : ga[b];
    }
    // m[] of blocks [16q, 16q + 16) as 4 little-endian words
    CDC_HD void m16(uint64_t q, uint32_t w[4]) const {
        const uint64_t b = q << 4, r = b - wb0;
        const uint8_t* p = (b >= wb0 && r + 16 <= wn) ? sm + r : gm + b;
#if defined(__CUDA_ARCH__)
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
#else
        const uint32_t* pw = reinterpret_cast<const uint32_t*>(p);
        for (int k = 0; k < 4; k++) w[k] = pw[k];
#endif
    }
    // m[] of blocks [4wi, 4wi + 4) as one little-endian word
    CDC_HD uint32_t m4(uint64_t wi) const {
        uint64_t b = wi << 2, r = b - wb0;
        if (b >= wb0 && r + 4 <= wn) return *reinterpret_cast<const uint32_t*>(sm + r);
        return *reinterpret_cast<const uint32_t*>(gm + b);
    }
};

struct Prm {
    uint32_t w, mn, mx;
};

// ---- raw helpers over any span [a, b), a < b (word at a time; the byte rules) --

CDC_HD uint32_t raw_max_span(const RawView& R, uint64_t a, uint64_t b) {
    uint32_t acc = 0;
    for (uint64_t wi = a >> 2, we = (b + 3) >> 2; wi < we; wi++)
        acc = vmax4(acc, clip_word(R.word(wi), wi, a, b));
    return hmax4(acc);
}

// first position in [a, b) whose byte is >= M (M >= 1); b if none
CDC_HD uint64_t raw_first_geq_span(const RawView& R, uint64_t a, uint64_t b, uint32_t M, uint32_t* val) {
    uint32_t Mx = M * 0x01010101u;
    for (uint64_t wi = a >> 2, we = (b + 3) >> 2; wi < we; wi++) {
        uint32_t v = R.word(wi);
        uint32_t h = clip_word(vcmpge4(v, Mx), wi, a, b);
        if (h) {
            uint32_t k = (uint32_t)((ffs32(h) - 1) >> 3);
            *val = (v >> (8 * k)) & 0xFFu;
            return (wi << 2) + k;
        }
    }
    return b;
}

// ---- raw helpers inside one 64-byte block (a < b <= end of a's block): the
// granules are loaded together, then scanned in registers ---------------------

CDC_HD uint32_t raw_max(const RawView& R, uint64_t a, uint64_t b) {
    uint32_t w[16];
    R.block(a, b, w);
    const uint64_t b0 = a & ~63ull;
    const uint32_t oa = (uint32_t)(a - b0), ob = (uint32_t)(b - b0);
    ByteMax m;
    CDC_UNROLL
    for (uint32_t i = 0; i < 16; i++) m.add(clip_in_block(w[i], i, oa, ob));
    return m.get();
}

// first position in [a, b) whose byte is >= M (M >= 1); b if none
CDC_HD uint64_t raw_first_geq(const RawView& R, uint64_t a, uint64_t b, uint32_t M, uint32_t* val) {
    uint32_t w[16];
    R.block(a, b, w);
    const uint64_t b0 = a & ~63ull;
    const uint32_t oa = (uint32_t)(a - b0), ob = (uint32_t)(b - b0), K = ge_key(M);
    CDC_UNROLL
    for (uint32_t i = 0; i < 16; i++) {
        const uint32_t f = ge_flags(clip_in_block(w[i], i, oa, ob), K);
        if (f) {
            const uint32_t k = (uint32_t)((ffs32(f) - 1) >> 3);
            *val = (w[i] >> (8 * k)) & 0xFFu;
            return b0 + 4 * i + k;
        }
    }
    return b;
}

// maximum of [a, b) and the position of its first occurrence (one block)
CDC_HD void raw_max_first(const RawView& R, uint64_t a, uint64_t b, uint32_t* v, uint64_t* p) {
    uint32_t w[16];
    R.block(a, b, w);
    const uint64_t b0 = a & ~63ull;
    const uint32_t oa = (uint32_t)(a - b0), ob = (uint32_t)(b - b0);
    ByteMax m;
    CDC_UNROLL
    for (uint32_t i = 0; i < 16; i++) m.add(clip_in_block(w[i], i, oa, ob));
    const uint32_t M = m.get();
    *v = M;
    *p = a;
    if (M == 0) return;  // every byte is 0: the first is at a
    const uint32_t K = ge_key(M);
    CDC_UNROLL
    for (uint32_t i = 0; i < 16; i++) {
        const uint32_t f = ge_flags(clip_in_block(w[i], i, oa, ob), K);
        if (f) {
            *p = b0 + 4 * i + (uint32_t)((ffs32(f) - 1) >> 3);
            return;
        }
    }
}

// ---- summary helpers --------------------------------------------------------

// maximum of m[] over blocks [b0, b1), b0 < b1 (16 blocks per step)
CDC_HD uint32_t sum_max(const SumView& S, uint64_t b0, uint64_t b1) {
    ByteMax m;
    for (uint64_t q = b0 >> 4, qe = (b1 + 15) >> 4; q < qe; q++) {
        uint32_t w[4];
        S.m16(q, w);
        CDC_UNROLL
        for (int k = 0; k < 4; k++) m.add(clip_word(w[k], 4 * q + (uint64_t)k, b0, b1));
        if (m.full()) return 255;  // cannot grow further
    }
    return m.get();
}

// first block in [b0, b1) with m[] >= M (M >= 1); b1 if none
CDC_HD uint64_t sum_first_geq(const SumView& S, uint64_t b0, uint64_t b1, uint32_t M) {
    const uint32_t K = ge_key(M);
    for (uint64_t q = b0 >> 4, qe = (b1 + 15) >> 4; q < qe; q++) {
        uint32_t w[4];
        S.m16(q, w);
        CDC_UNROLL
        for (int k = 0; k < 4; k++) {
            const uint64_t wi = 4 * q + (uint64_t)k;
            const uint32_t f = ge_flags(clip_word(w[k], wi, b0, b1), K);
            if (f) return (wi << 2) + (uint32_t)((ffs32(f) - 1) >> 3);
        }
    }
    return b1;
}

// Extreme Byte Search: maximum byte of [a, b), a < b
CDC_HD uint32_t range_max(const SumView& S, const RawView& R, uint64_t a, uint64_t b) {
    uint64_t ba = a >> 6, bl = (b - 1) >> 6;
    if (ba == bl) {
        if ((a & 63) == 0 && (b & 63) == 0) return S.m(ba);
        if (S.m(ba) == 0) return 0;
        return raw_max(R, a, b);
    }
    uint64_t fb = (a + 63) >> 6, lb = b >> 6;  // whole blocks [fb, lb)
    uint32_t M = fb < lb ? sum_max(S, fb, lb) : 0;
    if ((a & 63) && S.m(ba) > M) {
        uint32_t h = raw_max(R, a, (ba + 1) << 6);
        if (h > M) M = h;
    }
    if ((b & 63) && S.m(bl) > M) {
        uint32_t t = raw_max(R, bl << 6, b);
        if (t > M) M = t;
    }
    return M;
}

// Range Scan (GEQ): first position in [from, to) with byte >= M (M >= 1);
// `to` if none. *val receives the byte found.
CDC_HD uint64_t first_geq(const SumView& S, const RawView& R, uint64_t from, uint64_t to,
                          uint32_t M, uint32_t* val) {
    uint64_t b = from >> 6;
    uint64_t bend = (to - 1) >> 6;  // last block touched
    if ((from & 63) != 0 || b == bend) {
        uint64_t bhi = (b + 1) << 6;
        uint32_t bm = S.m(b);
        if (bm >= M) {
            uint64_t a = (b << 6) + S.a(b);
            if (bm == M && a >= from) {
                // every byte >= M in this block equals M; the first is a
                if (a < to) { *val = M; return a; }
                return to;  // a >= to implies to <= bhi
            }
            uint64_t e = umin64(bhi, to);
            uint64_t r = raw_first_geq(R, from, e, M, val);
            if (r < e) return r;
        }
        if (b == bend) return to;
        b++;
    }
    while (b <= bend) {
        uint64_t bh = sum_first_geq(S, b, bend + 1, M);
        if (bh > bend) return to;
        uint64_t blo = bh << 6;
        uint32_t bm = S.m(bh);
        uint64_t a = blo + S.a(bh);
        if (bm == M) {
            if (a < to) { *val = M; return a; }
            return to;
        }
        uint64_t e = umin64(blo + 64, to);
        uint64_t r = raw_first_geq(R, blo, e, M, val);
        if (r < e) return r;
        if (e == to) return to;
        b = bh + 1;
    }
    return to;
}

// ---- the chunk rules ---------------------------------------------------------

// RAM (Section 2.1, Section 3.3).
CDC_HD uint64_t next_ram(const SumView& S, const RawView& R, const Prm& P, uint64_t fhi,
                         uint64_t s) {
    if (fhi - s <= P.w) return fhi;
    uint64_t limit = umin64(fhi, s + P.mx);
    uint64_t t = s + P.w;
    uint32_t M = range_max(S, R, s, t);
    uint64_t j0 = umax64(t, s + P.mn - 1);
    if (j0 >= limit) return limit;
    if (M == 0) return j0 + 1;
    uint32_t val;
    uint64_t j = first_geq(S, R, j0, limit, M, &val);
    return j < limit ? j + 1 : limit;
}

// AE-Max over the (possibly complemented) bytes, w >= 64 (Section 2.1,
// Section 3.3). p is the current target, v its value, cur the first byte not
// yet known to be <= v.
CDC_HD uint64_t next_ae(const SumView& S, const RawView& R, const Prm& P, uint64_t fhi,
                        uint64_t s) {
    uint64_t limit = umin64(fhi, s + P.mx);
    if (s + 1 >= limit) return limit;
    uint64_t p;
    uint32_t v;
    {
        uint64_t b = s >> 6;
        uint64_t a = (b << 6) + S.a(b);
        if (a >= s && a < limit) {
            p = a;
            v = S.m(b);
        } else {
            raw_max_first(R, s, umin64((b + 1) << 6, limit), &v, &p);
        }
    }
    uint64_t cur = p + 1;
    for (;;) {
        uint64_t t = umax64(p + P.w, s + P.mn - 1);
        if (t >= limit) return limit;
        if (v == 255) return t + 1;
        uint64_t to = t + 1;
        if (cur & 63) {
            uint64_t bc = cur >> 6, bhi = (bc + 1) << 6;
            uint32_t bm = S.m(bc);
            if (bm > v) {
                uint64_t a = (bc << 6) + S.a(bc);
                if (a >= cur && bhi <= to) {
                    p = a; v = bm; cur = a + 1;
                    continue;
                }
                uint64_t e = umin64(bhi, to);
                uint32_t val;
                uint64_t q = raw_first_geq(R, cur, e, v + 1, &val);
                if (q < e) {
                    p = q; v = val; cur = q + 1;
                    continue;
                }
            }
            if (bhi >= to) return to;
            cur = bhi;
        }
        uint64_t bf = cur >> 6, bl = (to - 1) >> 6;
        uint64_t bh = sum_first_geq(S, bf, bl + 1, v + 1);
        if (bh > bl) return to;
        uint64_t blo = bh << 6;
        if (blo + 64 <= to) {
            p = blo + S.a(bh); v = S.m(bh); cur = p + 1;
            continue;
        }
        uint32_t val;
        uint64_t q = raw_first_geq(R, blo, to, v + 1, &val);
        if (q < to) {
            p = q; v = val; cur = q + 1;
            continue;
        }
        return to;
    }
}

// MAXP from per-block targets (w >= 63: at most one target per block).
// Only targets whose windows lie inside the file [flo, fhi) count.
CDC_HD uint64_t next_maxp(const SumView& S, const Prm& P, uint64_t flo, uint64_t fhi,
                          uint64_t s) {
    uint64_t limit = umin64(fhi, s + P.mx);
    uint64_t cmin = umax64(s + P.mn - 1, flo + P.w);
    uint64_t cend = fhi > flo + P.w ? umin64(limit, fhi - P.w) : 0;
    if (cmin >= cend) return limit;
    uint64_t b0 = cmin >> 6, b1 = ((cend - 1) >> 6) + 1;
    for (uint64_t wi = b0 >> 2, we = (b1 + 3) >> 2; wi < we; wi++) {
        uint32_t v = S.m4(wi);
        if (v == 0xFFFFFFFFu) continue;
        for (uint32_t k = 0; k < 4; k++) {
            uint64_t bb = (wi << 2) + k;
            uint32_t o = (v >> (8 * k)) & 0xFFu;
            if (o == 0xFFu || bb < b0 || bb >= b1) continue;
            uint64_t c = (bb << 6) + o;
            if (c >= cmin && c < cend) return c + 1;
        }
    }
    return limit;
}

// ---- byte-level rules (no summaries): used for w below the block size and
// for cross-checking the summary path -------------------------------------------

CDC_HD uint64_t next_ram_bytes(const RawView& R, const Prm& P, uint64_t fhi, uint64_t s) {
    if (fhi - s <= P.w) return fhi;
    uint64_t limit = umin64(fhi, s + P.mx);
    uint64_t t = s + P.w;
    uint32_t M = raw_max_span(R, s, t);
    uint64_t j0 = umax64(t, s + P.mn - 1);
    if (j0 >= limit) return limit;
    if (M == 0) return j0 + 1;
    uint32_t val;
    uint64_t j = raw_first_geq_span(R, j0, limit, M, &val);
    return j < limit ? j + 1 : limit;
}

CDC_HD uint64_t next_ae_bytes(const RawView& R, const Prm& P, uint64_t fhi, uint64_t s) {
    uint64_t limit = umin64(fhi, s + P.mx);
    uint64_t p = s;
    uint32_t v = R.byte(s);
    uint64_t cur = s + 1;
    for (;;) {
        uint64_t t = umax64(p + P.w, s + P.mn - 1);
        if (t >= limit) return limit;
        if (v == 255) return t + 1;
        uint32_t val;
        uint64_t q = raw_first_geq_span(R, cur, t + 1, v + 1, &val);
        if (q > t) return t + 1;
        p = q; v = val; cur = q + 1;
    }
}

CDC_HD bool maxp_target_bytes(const RawView& R, uint64_t c, uint32_t w) {
    uint32_t v = R.byte(c);
    if (v == 0) return false;
    uint32_t lm = raw_max_span(R, c - w, c);
    if (lm >= v) return false;
    return raw_max_span(R, c + 1, c + 1 + w) < v;
}

CDC_HD uint64_t next_maxp_bytes(const RawView& R, const Prm& P, uint64_t flo, uint64_t fhi,
                                uint64_t s) {
    uint64_t limit = umin64(fhi, s + P.mx);
    uint64_t cmin = umax64(s + P.mn - 1, flo + P.w);
    uint64_t cend = fhi > flo + P.w ? umin64(limit, fhi - P.w) : 0;
    for (uint64_t c = cmin; c < cend; c++)
        if (maxp_target_bytes(R, c, P.w)) return c + 1;
    return limit;
}

// Which rule the chain stage runs.
enum Rule : int {
    RULE_RAM = 0,        // RAM over summaries
    RULE_AE = 1,         // AE over summaries (w >= 64)
    RULE_MAXP = 2,       // MAXP over per-block targets (w >= 63)
    RULE_RAM_BYTES = 3,
    RULE_AE_BYTES = 4,
    RULE_MAXP_BYTES = 5
};

template <int RULE>
CDC_HD uint64_t next_cut(const SumView& S, const RawView& R, const Prm& P, uint64_t flo,
                         uint64_t fhi, uint64_t s) {
    if (RULE == RULE_RAM) return next_ram(S, R, P, fhi, s);
    if (RULE == RULE_AE) return next_ae(S, R, P, fhi, s);
    if (RULE == RULE_MAXP) return next_maxp(S, P, flo, fhi, s);
    if (RULE == RULE_RAM_BYTES) return next_ram_bytes(R, P, fhi, s);
    if (RULE == RULE_AE_BYTES) return next_ae_bytes(R, P, fhi, s);
    return next_maxp_bytes(R, P, flo, fhi, s);
}

// ---- fast-forward over quiet stretches ----------------------------------------
//
// Inside a run of zero bytes (complemented 0xFF for AE-Min) RAM and AE cut
// every w+1 bytes: the window maximum is 0 and the byte after it is >= 0
// (RAM), no byte exceeds the target 0 (AE). Where MAXP has no target within
// [s+min-1, s+max) it cuts at s+max. advance() takes such steps in one go;
// every other step is next_cut().

// first position in [p, bound) whose byte is non-zero, skipping quiet
// superblocks and zero blocks by their summaries; bound if none
CDC_HD uint64_t first_nonzero(const SumView& S, const RawView& R, uint64_t p, uint64_t bound) {
    while (p < bound) {
        if ((p & 4095) == 0 && S.sup && p + 4096 <= bound && S.sup[p >> 12] == 0) {
            p += 4096;
            continue;
        }
        const uint64_t b = p >> 6, e = umin64(bound, (b + 1) << 6);
        if (S.m(b) != 0) {
            uint32_t val;
            uint64_t r = raw_first_geq(R, p, e, 1, &val);
            if (r < e) return r;
        }
        p = e;
    }
    return bound;
}

// first MAXP target c with c0 <= c < c1, skipping superblocks without one; c1 if none
CDC_HD uint64_t first_target(const SumView& S, uint64_t c0, uint64_t c1) {
    uint64_t p = c0;
    while (p < c1) {
        if ((p & 4095) == 0 && S.sup && p + 4096 <= c1 && S.sup[p >> 12] == 0) {
            p += 4096;
            continue;
        }
        const uint64_t b = p >> 6;
        const uint32_t o = S.m(b);
        if (o != 0xFFu) {
            const uint64_t c = (b << 6) + o;
            if (c >= p && c < c1) return c;
        }
        p = (b + 1) << 6;
    }
    return c1;
}

// One or more chain steps from s (< stop). Returns the next position e and
// sets *k >= 1, *d: the chain visits s, s+d, ..., s+(k-1)d (all < stop) and
// then e. Equals k applications of next_cut().
template <int RULE>
CDC_HD uint64_t advance(const SumView& S, const RawView& R, const Prm& P, uint64_t flo, uint64_t fhi, uint64_t s,
                        uint64_t stop, uint32_t* k, uint64_t* d) {
    if (RULE == RULE_RAM || RULE == RULE_AE) {
        const uint64_t w = P.w, st = w + 1;
        // quick test: the window's first and last blocks are all zero
        if (P.mn <= st && s + w < fhi && S.m(s >> 6) == 0 && S.m((s + w - 1) >> 6) == 0) {
            // steps i with s_i = s + i*st, s_i + w < z (window and cut byte zero),
            // s_i + w < fhi (not the tail) and s_i < stop
            const uint64_t kstop = (stop - 1 - s) / st + 1;
            const uint64_t kfhi = (fhi - 1 - s - w) / st + 1;
            uint64_t kmax = kstop < kfhi ? kstop : kfhi;
            const uint64_t z = first_nonzero(S, R, s, s + (kmax - 1) * st + w + 1);
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
        const uint64_t e1 = next_maxp(S, P, flo, fhi, s);
        if (e1 == s + P.mx && e1 < fhi) {
            // forced cut: later forced cuts until a window reaches the next target
            const uint64_t mx = P.mx;
            const uint64_t c0 = umax64(s + P.mn - 1, flo + P.w);
            const uint64_t cend = fhi > flo + P.w ? fhi - P.w : 0;
            const uint64_t kstop = (stop - 1 - s) / mx + 1;
            // forced cut s_i + mx must stay <= fhi: i <= (fhi - s - mx) / mx
            const uint64_t kfhi = (fhi - s) / mx;
            uint64_t kmax = kstop < kfhi ? kstop : kfhi;
            if (kmax >= 2) {
                const uint64_t lim = umin64(cend, s + kmax * mx);
                const uint64_t c = c0 < lim ? first_target(S, c0, lim) : lim;
                // step i is forced while its window [s_i+mn-1, s_i+mx) misses c: s_i + mx <= c
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
    const uint64_t e = next_cut<RULE>(S, R, P, flo, fhi, s);
    *k = 1;
    *d = e - s;
    return e;
}

// ---- block summaries (the summary kernel's per-block arithmetic, also used
// by the host check) ------------------------------------------------------------

// maximum and first position of the maximum of 64 bytes given as 16 words
CDC_HD void block_max_first(const uint32_t* wds, uint32_t* mx, uint32_t* first) {
    uint32_t acc = 0;
    for (int i = 0; i < 16; i++) acc = vmax4(acc, wds[i]);
    uint32_t M = hmax4(acc), Mx = M * 0x01010101u;
    for (int i = 0; i < 16; i++) {
        uint32_t e = vcmpeq4(wds[i], Mx);
        if (e) {
            *mx = M;
            *first = (uint32_t)(4 * i + ((ffs32(e) - 1) >> 3));
            return;
        }
    }
    *mx = M;
    *first = 0;
}

}  // namespace cdc
