/*
 * CPU oracle for hashless content-defined chunking: RAM, AE-Max, AE-Min, MAXP.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, sequential
 * statement of what the chunkers compute. Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it. It shares no code,
 * header, table or helper with the GPU library.
 *
 * Source: arxiv 2508.05797 ("VectorCDC"), Section 2.1 (the AE, MAXP and RAM
 * paragraphs) and Section 3.3 ("Putting it together"). The paper checks that
 * its vector versions produce chunks identical to the native algorithms
 * (Section 5.2, "Vector-acceleration Impact"); the GPU path is held to the
 * same standard against this file.
 *
 * Conventions (shared by all algorithms):
 *   - Bytes are unsigned 0..255 (the paper compares bytes as hexadecimal
 *     values, e.g. 0xE1 vs 0x21 in Section 3.1).
 *   - A chunk is [s, e); next(s) returns e. The chunker emits
 *     e_1 = next(0), e_2 = next(e_1), ..., the last one equal to len.
 *   - min / max bound the chunk size: no cut before s + min, a forced cut at
 *     s + max (the usual CDC rule of Section 2.1, hash-based paragraph). The
 *     final chunk ends at len and may be shorter than min.
 *
 * Readings of passages the paper leaves open (each is listed in the design
 * notes with its reason):
 *   RAM  : the cut goes right after the first byte at or beyond the window
 *          whose value is >= the window maximum (GEQ), and that byte belongs
 *          to the chunk. If no more than w bytes remain, the rest is one chunk.
 *   AE   : a new target needs a strictly greater byte (GT); a byte equal to
 *          the target inside the window does not block the cut; the cut goes
 *          right after the w-byte window that follows the target.
 *   MAXP : a target is strictly greater than every byte within distance w on
 *          both sides; both windows must lie inside [0, len); windows may
 *          reach back into the previous chunk (positional test); the cut goes
 *          right after the target.
 */
#include <stddef.h>
#include <stdint.h>

enum { OR_RAM = 0, OR_AE_MAX = 1, OR_MAXP = 2, OR_AE_MIN = 3 };

static uint64_t umin(uint64_t a, uint64_t b) { return a < b ? a : b; }
static uint64_t umax(uint64_t a, uint64_t b) { return a > b ? a : b; }

/* RAM (Section 2.1 "RAM"; Section 3.3: an extreme byte search over the window
 * followed by a GEQ range scan). */
uint64_t oracle_next_ram(const uint8_t* B, uint64_t len, uint64_t s,
                         uint32_t w, uint32_t mn, uint32_t mx) {
    if (len - s <= w) return len;
    /* Extreme Byte Search: maximum of the w-byte window at the chunk start. */
    uint8_t M = 0;
    for (uint64_t i = s; i < s + w; i++)
        if (B[i] > M) M = B[i];
    /* Range Scan (GEQ) from the first byte outside the window. */
    uint64_t limit = umin(len, s + mx);
    for (uint64_t j = umax(s + w, s + mn - 1); j < limit; j++)
        if (B[j] >= M) return j + 1;
    return limit;
}

/* AE (Section 2.1 "AE"; Section 3.3). dir = +1 for AE-Max, -1 for AE-Min.
 * p is the current target (extreme so far); the cut is placed after the
 * w-byte window that follows p once that window holds no byte beyond it. */
uint64_t oracle_next_ae(const uint8_t* B, uint64_t len, uint64_t s,
                        uint32_t w, uint32_t mn, uint32_t mx, int dir) {
    uint64_t limit = umin(len, s + mx);
    uint64_t p = s;
    for (uint64_t i = s + 1; i < limit; i++) {
        int beyond = dir > 0 ? (B[i] > B[p]) : (B[i] < B[p]);
        if (beyond)
            p = i;                                  /* new target */
        else if (i - p >= w && i + 1 - s >= mn)
            return i + 1;                           /* window after p is clear */
    }
    return limit;
}

/* MAXP local-maximum test (Section 2.1 "MAXP"): i is a target when both
 * w-byte windows around it lie inside [0, len) and every byte in them is
 * strictly smaller than B[i]. */
int oracle_maxp_is_target(const uint8_t* B, uint64_t len, uint64_t i, uint32_t w) {
    if (i < w || i + w >= len) return 0;
    for (uint64_t k = 1; k <= w; k++) {
        if (B[i - k] >= B[i]) return 0;
        if (B[i + k] >= B[i]) return 0;
    }
    return 1;
}

/* MAXP (Section 2.1 "MAXP"; Section 3.3: range scans for a target, each
 * followed by the two window searches). The cut goes right after the first
 * target c with c + 1 - s >= min; none before s + max forces a cut there. */
uint64_t oracle_next_maxp(const uint8_t* B, uint64_t len, uint64_t s,
                          uint32_t w, uint32_t mn, uint32_t mx) {
    uint64_t limit = umin(len, s + mx);
    for (uint64_t c = s + mn - 1; c < limit; c++)
        if (oracle_maxp_is_target(B, len, c, w)) return c + 1;
    return limit;
}

uint64_t oracle_next(int alg, const uint8_t* B, uint64_t len, uint64_t s,
                     uint32_t w, uint32_t mn, uint32_t mx) {
    switch (alg) {
    case OR_RAM:    return oracle_next_ram(B, len, s, w, mn, mx);
    case OR_AE_MAX: return oracle_next_ae(B, len, s, w, mn, mx, +1);
    case OR_AE_MIN: return oracle_next_ae(B, len, s, w, mn, mx, -1);
    case OR_MAXP:   return oracle_next_maxp(B, len, s, w, mn, mx);
    default:        return 0;
    }
}

/* Chunk the whole buffer from offset 0. Writes up to cap chunk ends (the
 * boundaries) to out and returns how many there are in total. */
uint64_t oracle_chunk(int alg, const uint8_t* B, uint64_t len,
                      uint32_t w, uint32_t mn, uint32_t mx,
                      uint64_t* out, uint64_t cap) {
    uint64_t s = 0, n = 0;
    while (s < len) {
        uint64_t e = oracle_next(alg, B, len, s, w, mn, mx);
        if (n < cap) out[n] = e;
        n++;
        s = e;
    }
    return n;
}

/* All MAXP targets in [0, len), in increasing order (up to cap written). */
uint64_t oracle_maxp_targets(const uint8_t* B, uint64_t len, uint32_t w,
                             uint64_t* out, uint64_t cap) {
    uint64_t n = 0;
    for (uint64_t i = 0; i < len; i++)
        if (oracle_maxp_is_target(B, len, i, w)) {
            if (n < cap) out[n] = i;
            n++;
        }
    return n;
}

/* Extreme Byte Search (Section 3.1): the maximum (op 0) or minimum (op 1)
 * byte of B[a, b) and the offset of its first occurrence; an empty range
 * gives 0 (maximum) or 255 (minimum) at a. Plain loop, one byte at a time. */
uint32_t oracle_ebs(int op, const uint8_t* B, uint64_t len, uint64_t a, uint64_t b, uint64_t* pos) {
    if (b > len) b = len;
    uint32_t best = op == 1 ? 255 : 0;
    *pos = a;
    int seen = 0;
    for (uint64_t i = a; i < b; i++) {
        const uint32_t v = B[i];
        if (!seen || (op == 1 ? v < best : v > best)) {
            best = v;
            *pos = i;
            seen = 1;
        }
    }
    return best;
}

/* Range Scan (Section 3.2): the first offset i in [a, b) whose byte compares
 * true against t with GT (0), LT (1), GEQ (2), LEQ (3) or EQ (4); b as given
 * if none (the range is clipped to len for reading). */
uint64_t oracle_rs(int cmp, const uint8_t* B, uint64_t len, uint64_t a, uint64_t b, uint32_t t) {
    const uint64_t e = b < len ? b : len;
    for (uint64_t i = a; i < e; i++) {
        const uint32_t v = B[i];
        int hit = 0;
        switch (cmp) {
        case 0: hit = v > t; break;
        case 1: hit = v < t; break;
        case 2: hit = v >= t; break;
        case 3: hit = v <= t; break;
        default: hit = v == t; break;
        }
        if (hit) return i;
    }
    return b;
}

/* Bytes each processing pattern reads while the chunks of B are found, as
 * Section 3.3 composes the algorithms (the paper reports these shares in its
 * byte-share figure). Chunk by chunk from s (e = its end, L = min(len, s + max)):
 *   RAM: one Extreme Byte Search over the w-byte window at s, then one GEQ
 *        Range Scan from max(s + w, s + min - 1) up to and including the byte
 *        it stops at (or up to L when it finds none); a tail of at most w
 *        bytes is one search over the rest.
 *   AE:  from the first target s: an Extreme Byte Search over the w bytes
 *        after the target (clipped at L - 1); if that window holds a byte
 *        beyond the target, a GT (LT for AE-Min) Range Scan from the target
 *        finds the next target (the bytes after the target up to it) and the
 *        search repeats; otherwise the chunk ends after the window. Defined
 *        for min <= w + 1, where the window end is always a permitted cut.
 *   MAXP: Range Scans with the GT comparator, each followed by two Extreme
 *        Byte Searches (Section 3.3), from p = max(s + min - 1, w) (the first
 *        position that may end the chunk with both windows inside the data):
 *        a search over the left window [p - w, p) gives its maximum L and the
 *        last position m holding it; every position up to m + w still has m
 *        in its left window, so a GT scan for a byte above L over
 *        [p, min(m + w + 1, end)) finds the first of them that beats its own
 *        left window (end = min(L_chunk, len - w)); if it finds one (q), a
 *        search over the right window (q, q + w] decides whether q is a
 *        target (the chunk ends after it) or the scan goes on from q + 1;
 *        if it finds none, the scan goes on from its end. Scans read the
 *        bytes up to and including the one they stop at.
 * Adds to *ebs and *rs; returns 0, -1 for AE with min > w + 1, or -2 if a
 * MAXP cut differs from oracle_next (a self-check of the procedure). */
int oracle_byte_shares(int alg, const uint8_t* B, uint64_t len, uint32_t w, uint32_t mn, uint32_t mx,
                       uint64_t* ebs, uint64_t* rs) {
    if ((alg == OR_AE_MAX || alg == OR_AE_MIN) && mn > w + 1) return -1;
    uint64_t s = 0;
    while (s < len) {
        const uint64_t L = umin(len, s + mx);
        uint64_t e;
        if (alg == OR_MAXP) {
            const uint64_t cend = len > w ? umin(L, len - w) : 0;
            uint64_t p = umax(s + mn - 1, w);
            e = L;
            while (p < cend) {
                uint32_t lmax = 0;
                uint64_t m = p - w;
                for (uint64_t i = p - w; i < p; i++)  /* left window: maximum, last position */
                    if (B[i] >= lmax) {
                        lmax = B[i];
                        m = i;
                    }
                *ebs += w;
                const uint64_t stop = umin(cend, m + w + 1);
                const uint64_t q = oracle_rs(0, B, len, p, stop, lmax);
                if (q >= stop) {
                    *rs += stop - p;
                    p = stop;
                    continue;
                }
                *rs += q - p + 1;
                uint64_t at;
                const uint32_t rmax = oracle_ebs(0, B, len, q + 1, q + w + 1, &at);
                *ebs += w;
                if (B[q] > rmax) {
                    e = q + 1;
                    break;
                }
                p = q + 1;
            }
            if (e != oracle_next(alg, B, len, s, w, mn, mx)) return -2;
        } else if (alg == OR_RAM) {
            if (len - s <= w) {
                *ebs += len - s;
                e = len;
            } else {
                uint64_t at;
                const uint32_t M = oracle_ebs(0, B, len, s, s + w, &at);
                *ebs += w;
                const uint64_t from = mn - 1 > w ? s + mn - 1 : s + w;  /* the scan's first byte */
                if (from >= L) {
                    e = L;
                } else {
                    const uint64_t j = oracle_rs(2, B, len, from, L, M);
                    e = j < L ? j + 1 : L;
                    *rs += e - from;
                }
            }
        } else {
            const int op = alg == OR_AE_MIN ? 1 : 0;     /* window search for max or min */
            const int cmp = alg == OR_AE_MIN ? 1 : 0;    /* GT or LT */
            uint64_t p = s;
            for (;;) {
                const uint64_t wend = umin(p + w, L - 1);  /* window (p, wend] */
                uint64_t at;
                const uint32_t x = oracle_ebs(op, B, len, p + 1, wend + 1, &at);
                *ebs += wend - p;
                const int beyond = wend > p && (op ? x < B[p] : x > B[p]);
                if (!beyond) {
                    e = p + w < L ? p + w + 1 : L;
                    break;
                }
                const uint64_t r = oracle_rs(cmp, B, len, p + 1, wend + 1, B[p]);
                *rs += r - p;
                p = r;
            }
        }
        s = e;
    }
    return 0;
}

