// Test-only host build of the chain stage's per-thread chunk rules
// (paper_2508_05797_gb300/csrc/chain_logic.cuh), so that the summary-based
// rules can be compared with the CPU oracle without a GPU.
#include <vector>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "chain_logic.cuh"

using namespace cdc;

extern "C" uint64_t hc_next(int rule, const uint8_t* base, const uint8_t* smax, const uint8_t* sarg,
                            uint64_t wb0, uint64_t wn, const uint8_t* wm, const uint8_t* wa, uint32_t inv,
                            uint32_t w, uint32_t mn, uint32_t mx, uint64_t flo, uint64_t fhi, uint64_t s) {
    SumView S{smax, sarg, wm, wa, wb0, wn, nullptr};
    RawView R{base, inv};
    Prm P{w, mn, mx};
    switch (rule) {
    case RULE_RAM: return next_cut<RULE_RAM>(S, R, P, flo, fhi, s);
    case RULE_AE: return next_cut<RULE_AE>(S, R, P, flo, fhi, s);
    case RULE_MAXP: return next_cut<RULE_MAXP>(S, R, P, flo, fhi, s);
    case RULE_RAM_BYTES: return next_cut<RULE_RAM_BYTES>(S, R, P, flo, fhi, s);
    case RULE_AE_BYTES: return next_cut<RULE_AE_BYTES>(S, R, P, flo, fhi, s);
    default: return next_cut<RULE_MAXP_BYTES>(S, R, P, flo, fhi, s);
    }
}

// chain of one file [flo, fhi): returns the number of boundaries, writes up to cap
extern "C" uint64_t hc_chain(int rule, const uint8_t* base, const uint8_t* smax, const uint8_t* sarg, uint32_t inv,
                             uint32_t w, uint32_t mn, uint32_t mx, uint64_t flo, uint64_t fhi, uint64_t* out,
                             uint64_t cap) {
    uint64_t s = flo, n = 0;
    while (s < fhi) {
        s = hc_next(rule, base, smax, sarg, 0, 0, nullptr, nullptr, inv, w, mn, mx, flo, fhi, s);
        if (n < cap) out[n] = s - flo;
        n++;
    }
    return n;
}

extern "C" void hc_block_max_first(const uint8_t* block64, uint32_t* mx, uint32_t* first) {
    uint32_t wds[16];
    memcpy(wds, block64, 64);
    block_max_first(wds, mx, first);
}

// chain of one file with the multi-step advance(); sup: superblock summaries
extern "C" uint64_t hc_chain_adv(int rule, const uint8_t* base, const uint8_t* smax, const uint8_t* sarg,
                                 const uint8_t* sup, uint32_t inv, uint32_t w, uint32_t mn, uint32_t mx, uint64_t flo,
                                 uint64_t fhi, uint64_t stop_every, uint64_t* out, uint64_t cap, uint64_t* jumps) {
    SumView S{smax, sarg, nullptr, nullptr, 0, 0, sup};
    RawView R{base, inv};
    Prm P{w, mn, mx};
    uint64_t s = flo, n = 0, nj = 0;
    while (s < fhi) {
        uint64_t stop = stop_every ? umin64(fhi, (s / stop_every + 1) * stop_every) : fhi;
        uint32_t k;
        uint64_t d, e;
        switch (rule) {
        case RULE_RAM: e = advance<RULE_RAM>(S, R, P, flo, fhi, s, stop, &k, &d); break;
        case RULE_AE: e = advance<RULE_AE>(S, R, P, flo, fhi, s, stop, &k, &d); break;
        default: e = advance<RULE_MAXP>(S, R, P, flo, fhi, s, stop, &k, &d); break;
        }
        if (k > 1) nj++;
        for (uint32_t i = 1; i < k; i++) {
            if (n < cap) out[n] = s + i * d - flo;
            n++;
        }
        if (n < cap) out[n] = e - flo;
        n++;
        s = e;
    }
    *jumps = nj;
    return n;
}

// ---- candidate-graph rules (graph_logic.cuh) ------------------------------------

#include "graph_logic.cuh"

template <typename F>
static uint64_t with_rule(int rule, F f) {
    switch (rule) {
    case RULE_RAM: return f(std::integral_constant<int, RULE_RAM>{});
    case RULE_AE: return f(std::integral_constant<int, RULE_AE>{});
    default: return f(std::integral_constant<int, RULE_MAXP>{});
    }
}

// every candidate of the data [lo, hi) in increasing order, found block by
// block with block_cands(); returns the count, writes up to cap positions
extern "C" uint64_t hc_cands(int rule, const uint8_t* base, const uint8_t* smax, const uint8_t* sarg,
                             const uint8_t* sup, uint32_t inv, uint32_t w, uint32_t mn, uint32_t mx, uint64_t lo,
                             uint64_t hi, uint64_t* out, uint64_t cap) {
    SumView S{smax, sarg, nullptr, nullptr, 0, 0, sup};
    RawView R{base, inv};
    Prm P{w, mn, mx};
    return with_rule(rule, [&](auto rc) -> uint64_t {
        constexpr int RU = decltype(rc)::value;
        uint64_t qa, qb, n = 0;
        cand_source_range<RU>(P, lo, hi, &qa, &qb);
        const uint64_t sh = cand_shift<RU>(P);
        for (uint64_t b = qa >> 6; qa < qb && b <= (qb - 1) >> 6; b++) {
            uint64_t m = block_cands<RU>(S, R, P, b, qa, qb);
            while (m) {
                const int o = __builtin_ctzll(m);
                m &= m - 1;
                if (n < cap) out[n] = (b << 6) + (uint64_t)o + sh;
                n++;
            }
        }
        return n;
    });
}

extern "C" int hc_is_cand(int rule, const uint8_t* base, const uint8_t* smax, const uint8_t* sarg,
                          const uint8_t* sup, uint32_t inv, uint32_t w, uint32_t mn, uint32_t mx, uint64_t lo,
                          uint64_t hi, uint64_t y) {
    SumView S{smax, sarg, nullptr, nullptr, 0, 0, sup};
    RawView R{base, inv};
    Prm P{w, mn, mx};
    return (int)with_rule(rule, [&](auto rc) -> uint64_t {
        return is_cand<decltype(rc)::value>(S, R, P, lo, hi, y) ? 1 : 0;
    });
}

extern "C" uint64_t hc_cand_next(int rule, const uint8_t* base, const uint8_t* smax, const uint8_t* sarg,
                                 const uint8_t* sup, uint32_t inv, uint32_t w, uint32_t mn, uint32_t mx, uint64_t lo,
                                 uint64_t hi, uint64_t y, uint32_t* n) {
    SumView S{smax, sarg, nullptr, nullptr, 0, 0, sup};
    RawView R{base, inv};
    Prm P{w, mn, mx};
    return with_rule(rule, [&](auto rc) -> uint64_t {
        return cand_next<decltype(rc)::value>(S, R, P, lo, hi, y, n);
    });
}

// the chain of [lo, hi) as the candidate graph gives it: F from the start,
// candidate after candidate; the chunk ends between two candidates are taken
// by advance() again. Returns the count, writes up to cap ends (from lo).
extern "C" uint64_t hc_graph_chain(int rule, const uint8_t* base, const uint8_t* smax, const uint8_t* sarg,
                                   const uint8_t* sup, uint32_t inv, uint32_t w, uint32_t mn, uint32_t mx,
                                   uint64_t lo, uint64_t hi, uint64_t* out, uint64_t cap) {
    SumView S{smax, sarg, nullptr, nullptr, 0, 0, sup};
    RawView R{base, inv};
    Prm P{w, mn, mx};
    return with_rule(rule, [&](auto rc) -> uint64_t {
        constexpr int RU = decltype(rc)::value;
        uint64_t y = lo, n = 0;
        while (y < hi) {
            uint32_t c = 0;
            const uint64_t e = cand_next<RU>(S, R, P, lo, hi, y, &c);
            uint64_t s = y;
            for (uint32_t i = 0; i < c;) {
                uint32_t k;
                uint64_t d;
                const uint64_t e2 = advance<RU>(S, R, P, lo, hi, s, hi, &k, &d);
                for (uint32_t t = 1; t <= k; t++, i++) {
                    if (n < cap) out[n] = s + t * d - lo;
                    n++;
                }
                s = e2;
            }
            if (s != e) return ~0ull;  // the re-walk must land on F(y)
            y = e;
        }
        return n;
    });
}

// the graph's chain with the running maxima inside superblocks (pre, suf)
extern "C" uint64_t hc_graph_chain_t(int rule, const uint8_t* base, const uint8_t* smax, const uint8_t* sarg,
                                     const uint8_t* sup, uint32_t inv, uint32_t w, uint32_t mn, uint32_t mx,
                                     uint64_t lo, uint64_t hi, const uint8_t* pre, const uint8_t* suf,
                                     uint64_t* out, uint64_t cap) {
    SumView S{smax, sarg, nullptr, nullptr, 0, 0, sup};
    RawView R{base, inv};
    Prm P{w, mn, mx};
    PreSuf T{pre, suf};
    return with_rule(rule, [&](auto rc) -> uint64_t {
        constexpr int RU = decltype(rc)::value;
        uint64_t y = lo, n = 0;
        while (y < hi) {
            uint32_t c = 0;
            const uint64_t e = cand_next_t<RU>(S, T, R, P, lo, hi, y, &c);
            uint64_t s = y;
            for (uint32_t i = 0; i < c;) {
                uint32_t k;
                uint64_t d;
                const uint64_t e2 = advance<RU>(S, R, P, lo, hi, s, hi, &k, &d);
                for (uint32_t t = 1; t <= k; t++, i++) {
                    if (n < cap) out[n] = s + t * d - lo;
                    n++;
                }
                s = e2;
            }
            if (s != e) return ~0ull;
            y = e;
        }
        return n;
    });
}


// F of every candidate of [lo, hi) from the whole candidate list (cover = hi):
// writes the list index or ~0u (the list cannot decide) per candidate, and
// checks each decided one against cand_next(); returns the number decided, or
// ~0ull - i if candidate i disagrees
extern "C" uint64_t hc_list_check(int rule, const uint8_t* base, const uint8_t* smax, const uint8_t* sarg,
                                  const uint8_t* sup, uint32_t inv, uint32_t w, uint32_t mn, uint32_t mx, uint64_t lo,
                                  uint64_t hi, const uint32_t* pos, const uint8_t* val, uint32_t n, uint64_t lbase,
                                  uint32_t* out) {
    SumView S{smax, sarg, nullptr, nullptr, 0, 0, sup};
    RawView R{base, inv};
    Prm P{w, mn, mx};
    PreSuf T{nullptr, nullptr};
    // group maxima of the list, as the local kernel builds them
    std::vector<uint8_t> gm((n + 31) / 32, 0);
    for (uint32_t i = 0; i < n; i++) gm[i / 32] = val[i] > gm[i / 32] ? val[i] : gm[i / 32];
    CandList L{pos, val, n, lbase, hi, gm.data()};
    WMaxSum wm{&S, &T, &R};
    return with_rule(rule, [&](auto rc) -> uint64_t {
        constexpr int RU = decltype(rc)::value;
        uint64_t decided = 0;
        for (uint32_t i = 0; i < n; i++) {
            const uint64_t y = lbase + pos[i];
            uint32_t lc = 0;
            const uint32_t k = list_next<RU>(L, wm, R, P, lo, hi, y, &lc);
            out[i] = k;
            if (k == LIST_GENERIC) continue;
            uint32_t c = 0;
            const uint64_t e = cand_next<RU>(S, R, P, lo, hi, y, &c);
            if (c != lc || e != lbase + pos[k]) return ~0ull - i;
            decided++;
        }
        return decided;
    });
}
