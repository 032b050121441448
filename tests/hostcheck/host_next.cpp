// Test-only host build of the chain stage's per-thread chunk rules
// (paper_2508_05797_gb300/csrc/chain_logic.cuh), so that the summary-based
// rules can be compared with the CPU oracle without a GPU.
#include <stdint.h>
#include <string.h>

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
