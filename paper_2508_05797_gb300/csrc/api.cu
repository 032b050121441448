// api.cu -- the C ABI (include/cdc.h): handles, workspace, validation and the
// launch sequence  [batch set-up] -> summaries (or control reset) -> chain.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "../../include/cdc.h"
#include "cdc_device.cuh"
#include "cdc_launch.h"
#include "graph_logic.cuh"

using namespace cdc;

struct cdc_handle_s {
    int device = 0;
    int sm_count = 0;
    // workspace (grow-only)
    uint8_t* smax = nullptr;
    uint8_t* sarg = nullptr;
    size_t sum_cap = 0;  // bytes of smax
    size_t sarg_cap = 0;
    uint8_t* ssup = nullptr;
    size_t ssup_cap = 0;
    uint8_t* st = nullptr;  // SegState array
    size_t st_cap = 0;      // bytes
    uint8_t* groups = nullptr;  // GroupState array
    size_t groups_cap = 0;      // bytes
    uint8_t* hash = nullptr;    // per-segment position hashes
    size_t hash_cap = 0;        // bytes
    uint8_t* plog = nullptr;    // per-segment step logs
    size_t plog_cap = 0;        // bytes
    Ctrl* ctrl = nullptr;
    uint64_t* item_off = nullptr;
    uint64_t* scan_tmp = nullptr;
    size_t scan_cap = 0;
    size_t files_cap = 0;
    uint32_t* item_file = nullptr;
    size_t item_file_cap = 0;
    uint8_t* host_stage = nullptr;  // cdc_chunk_host device copies
    size_t host_stage_cap = 0;
    uint64_t* host_out = nullptr;
    size_t host_out_cap = 0;
    Ctrl* pinned_ctrl = nullptr;  // page-locked copy of the control block
    // candidate-graph chain stage (graph.cu)
    uint32_t* g_cpos = nullptr;
    size_t g_cpos_cap = 0;
    uint32_t* g_cft = nullptr;
    size_t g_cft_cap = 0;
    uint32_t* g_csc = nullptr;
    size_t g_csc_cap = 0;
    unsigned long long* g_cex = nullptr;
    size_t g_cex_cap = 0;
    uint32_t* g_cnum = nullptr;
    size_t g_cnum_cap = 0;
    uint32_t* g_sent = nullptr;
    size_t g_sent_cap = 0;
    uint64_t* g_soff = nullptr;
    size_t g_soff_cap = 0;
    unsigned long long* g_uex = nullptr;
    size_t g_uex_cap = 0;
    uint32_t* g_uent = nullptr;
    size_t g_uent_cap = 0;
    uint64_t* g_uoff = nullptr;
    size_t g_uoff_cap = 0;
    uint8_t* g_spre = nullptr;
    size_t g_spre_cap = 0;
    uint8_t* g_ssuf = nullptr;
    size_t g_ssuf_cap = 0;
    uint8_t* g_cval = nullptr;
    size_t g_cval_cap = 0;
    unsigned long long* g_ticket = nullptr;
    size_t g_ticket_cap = 0;
    uint8_t* g_cfar = nullptr;
    size_t g_cfar_cap = 0;
    uint32_t* g_far = nullptr;
    size_t g_far_cap = 0;
    // options
    int64_t seg = 0, span = 0, timeout_ms = 2000, force_bytes = 0, hold_item = -1, stats = 0, warp_chains = 0;
    int64_t starts = 0;
    int64_t pipeline = 0, graph_seg = 0, graph_cap = 0;
    // last-call bookkeeping
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // start, summaries done, end, speculation done
    bool timed = false;
    int launches = 0;
    int stage = 0;  // chain stage of the last single-stream call: 1 speculation, 2 candidate graph
    // profiling ring: 4 events (as ev[]) for each of up to PROF_CAP calls
    static constexpr int PROF_CAP = 1024;
    int64_t profile = 0;
    cudaEvent_t* prof_ev = nullptr;
    int prof_n = 0;
    int64_t prof_launches = 0;
    cudaEvent_t* last_ev = nullptr;
};

static const char* kStatusNames[] = {"CDC_OK", "CDC_ERR_INVALID", "CDC_ERR_CAPACITY", "CDC_ERR_CUDA",
                                     "CDC_ERR_TIMEOUT", "CDC_ERR_NOMEM", "CDC_ERR_INTERNAL"};

extern "C" const char* cdc_status_string(cdc_status s) {
    if ((int)s >= 0 && (int)s < 7) return kStatusNames[(int)s];
    return "CDC_ERR_UNKNOWN";
}

static bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

template <typename T>
static cdc_status grow(T** p, size_t* cap, size_t need, bool zero, cudaStream_t s) {
    if (*cap >= need && *p) return CDC_OK;
    if (capturing(s)) return CDC_ERR_NOMEM;
    size_t n = need + need / 4 + 64;
    if (*p) {
        cudaStreamSynchronize(s);
        cudaFree(*p);
        *p = nullptr;
        *cap = 0;
    }
    T* q = nullptr;
    if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return CDC_ERR_NOMEM;
    }
    if (zero && cudaMemset(q, 0, n * sizeof(T)) != cudaSuccess) {
        cudaFree(q);
        return CDC_ERR_CUDA;
    }
    *p = q;
    *cap = n;
    return CDC_OK;
}

extern "C" cdc_status cdc_create(cdc_handle* out, int device) {
    if (!out) return CDC_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return CDC_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return CDC_ERR_CUDA;
    cdc_handle h = new cdc_handle_s();
    h->device = device;
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&h->ctrl, sizeof(Ctrl)) != cudaSuccess || cudaMemset(h->ctrl, 0, sizeof(Ctrl)) != cudaSuccess ||
        cudaMallocHost(&h->pinned_ctrl, sizeof(Ctrl)) != cudaSuccess) {
        cudaGetLastError();
        cdc_destroy(h);
        return CDC_ERR_NOMEM;
    }
    for (int i = 0; i < 4; i++) cudaEventCreate(&h->ev[i]);
    *out = h;
    return CDC_OK;
}

extern "C" cdc_status cdc_destroy(cdc_handle h) {
    if (!h) return CDC_OK;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    cudaFree(h->smax);
    cudaFree(h->sarg);
    cudaFree(h->ssup);
    cudaFree(h->groups);
    cudaFree(h->hash);
    cudaFree(h->plog);
    cudaFree(h->st);
    cudaFree(h->ctrl);
    cudaFree(h->item_off);
    cudaFree(h->scan_tmp);
    cudaFree(h->item_file);
    cudaFree(h->host_stage);
    cudaFree(h->host_out);
    cudaFree(h->g_cpos);
    cudaFree(h->g_cft);
    cudaFree(h->g_csc);
    cudaFree(h->g_cex);
    cudaFree(h->g_cnum);
    cudaFree(h->g_sent);
    cudaFree(h->g_soff);
    cudaFree(h->g_uex);
    cudaFree(h->g_uent);
    cudaFree(h->g_uoff);
    cudaFree(h->g_spre);
    cudaFree(h->g_ssuf);
    cudaFree(h->g_cval);
    cudaFree(h->g_ticket);
    cudaFree(h->g_cfar);
    cudaFree(h->g_far);
    if (h->pinned_ctrl) cudaFreeHost(h->pinned_ctrl);
    for (int i = 0; i < 4; i++)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    if (h->prof_ev) {
        for (int i = 0; i < 4 * cdc_handle_s::PROF_CAP; i++) cudaEventDestroy(h->prof_ev[i]);
        free(h->prof_ev);
    }
    cudaGetLastError();
    delete h;
    return CDC_OK;
}

extern "C" cdc_status cdc_set_option(cdc_handle h, cdc_option opt, int64_t v) {
    if (!h) return CDC_ERR_INVALID;
    switch (opt) {
    case CDC_OPT_SEGMENT:
        if (v < 0 || v > (1ll << 24) || (v && v < 64)) return CDC_ERR_INVALID;
        h->seg = v;
        return CDC_OK;
    case CDC_OPT_SPAN:
        if (v < 0) return CDC_ERR_INVALID;
        h->span = v;
        return CDC_OK;
    case CDC_OPT_TIMEOUT_MS:
        if (v <= 0) return CDC_ERR_INVALID;
        h->timeout_ms = v;
        return CDC_OK;
    case CDC_OPT_FORCE_BYTES: h->force_bytes = v ? 1 : 0; return CDC_OK;
    case CDC_OPT_DEBUG_HOLD_ITEM: h->hold_item = v; return CDC_OK;
    case CDC_OPT_STATS:
        h->stats = v ? 1 : 0;
        return CDC_OK;
    case CDC_OPT_WARP_CHAINS:
        if (v < 0 || v > NL) return CDC_ERR_INVALID;
        h->warp_chains = v;
        return CDC_OK;
    case CDC_OPT_STARTS:
        if (v < 0 || v > NL) return CDC_ERR_INVALID;
        h->starts = v;
        return CDC_OK;
    case CDC_OPT_PIPELINE:
        if (v < 0 || v > 2) return CDC_ERR_INVALID;
        h->pipeline = v;
        return CDC_OK;
    case CDC_OPT_GRAPH_SEGMENT:
        if (v < 0 || v > (1ll << 26) || (v & 4095)) return CDC_ERR_INVALID;
        h->graph_seg = v;
        return CDC_OK;
    case CDC_OPT_GRAPH_SLOTS:
        if (v < 0 || v > 4096) return CDC_ERR_INVALID;
        h->graph_cap = v;
        return CDC_OK;
    case CDC_OPT_PROFILE:
        if (v && !h->prof_ev) {
            cudaSetDevice(h->device);
            h->prof_ev = (cudaEvent_t*)calloc(4 * cdc_handle_s::PROF_CAP, sizeof(cudaEvent_t));
            if (!h->prof_ev) return CDC_ERR_NOMEM;
            for (int i = 0; i < 4 * cdc_handle_s::PROF_CAP; i++)
                if (cudaEventCreate(&h->prof_ev[i]) != cudaSuccess) return CDC_ERR_CUDA;
        }
        h->profile = v ? 1 : 0;
        h->prof_n = 0;
        h->prof_launches = 0;
        return CDC_OK;
    default: return CDC_ERR_INVALID;
    }
}

extern "C" cdc_status cdc_get_option(cdc_handle h, cdc_option opt, int64_t* v) {
    if (!h || !v) return CDC_ERR_INVALID;
    switch (opt) {
    case CDC_OPT_SEGMENT: *v = h->seg; return CDC_OK;
    case CDC_OPT_SPAN: *v = h->span; return CDC_OK;
    case CDC_OPT_TIMEOUT_MS: *v = h->timeout_ms; return CDC_OK;
    case CDC_OPT_FORCE_BYTES: *v = h->force_bytes; return CDC_OK;
    case CDC_OPT_DEBUG_HOLD_ITEM: *v = h->hold_item; return CDC_OK;
    case CDC_OPT_PROFILE: *v = h->profile; return CDC_OK;
    case CDC_OPT_STATS: *v = h->stats; return CDC_OK;
    case CDC_OPT_WARP_CHAINS: *v = h->warp_chains; return CDC_OK;
    case CDC_OPT_STARTS: *v = h->starts; return CDC_OK;
    case CDC_OPT_PIPELINE: *v = h->pipeline; return CDC_OK;
    case CDC_OPT_GRAPH_SEGMENT: *v = h->graph_seg; return CDC_OK;
    case CDC_OPT_GRAPH_SLOTS: *v = h->graph_cap; return CDC_OK;
    default: return CDC_ERR_INVALID;
    }
}

static bool valid_params(cdc_alg alg, cdc_params p) {
    if ((int)alg < 0 || (int)alg > 3) return false;
    if (p.w < 1 || p.min < 1 || p.min > p.max) return false;
    if (alg != CDC_MAXP && p.w >= p.max) return false;
    return true;
}

// which summaries and which chain rule a call uses
struct Plan {
    int sum;   // SumKind
    int rule;  // Rule
    uint32_t inv;
    uint32_t halo;
};

static constexpr uint32_t MAXP_SUMMARY_MAX_W = 16384;
static constexpr uint32_t kLogCap = HANDLE_LOG_CAP;

static Plan make_plan(cdc_handle h, cdc_alg alg, cdc_params p) {
    Plan pl{SUM_NONE, RULE_RAM_BYTES, 0u, 0u};
    bool bytes = h->force_bytes != 0;
    switch (alg) {
    case CDC_RAM:
        if (!bytes) { pl.sum = SUM_MAX; pl.rule = RULE_RAM; }
        else pl.rule = RULE_RAM_BYTES;
        break;
    case CDC_AE:
    case CDC_AE_MIN:
        pl.inv = alg == CDC_AE_MIN ? 0xFFFFFFFFu : 0u;
        if (!bytes && p.w >= 64) {
            pl.sum = alg == CDC_AE_MIN ? SUM_MAX_INV : SUM_MAX;
            pl.rule = RULE_AE;
        } else pl.rule = RULE_AE_BYTES;
        break;
    case CDC_MAXP:
        if (!bytes && p.w >= 63 && p.w <= MAXP_SUMMARY_MAX_W) {
            pl.sum = SUM_MAXP;
            pl.rule = RULE_MAXP;
            pl.halo = maxp_halo_blocks(p.w);
        } else pl.rule = RULE_MAXP_BYTES;
        break;
    }
    return pl;
}

// segment size: a few segments per SM (four for RAM / AE, sixteen for MAXP),
// 64-byte multiple. Longer segments let more speculative chains join inside
// them; the cap keeps the staged summary window (segment + bound room + max,
// two bytes per block for RAM / AE, one for MAXP) small enough for five or six
// resident speculation blocks per SM. Caps measured on the 4 GiB mixed stream:
// 384 KiB for RAM / AE up to max = 64 KiB, 256 KiB above, 512 KiB for MAXP.
// Floors measured on 16 MiB inputs: 32 KiB for RAM / AE, 64 KiB for MAXP (15%
// faster than 32 KiB). Four per SM rather than sixteen for RAM / AE: on the
// mixed stream 1.45x (RAM) and 1.24x (AE) faster at 64 MiB, 1.18x at 256 MiB,
// the same at 16 MiB and 1 GiB; MAXP gained 7% at 64-256 MiB but lost 8% at
// 1 GiB, so it keeps sixteen.
static uint64_t pick_seg(cdc_handle h, cdc_alg alg, cdc_params p, uint64_t len, uint64_t n_files) {
    if (h->seg) return (uint64_t)h->seg;
    const uint64_t cap = alg == CDC_MAXP ? (512u << 10) : p.max >= (128u << 10) ? (256u << 10) : (384u << 10);
    const uint64_t floor = alg == CDC_MAXP ? (64u << 10) : (32u << 10);
    const uint64_t per_sm = alg == CDC_MAXP ? 16 : 4;
    uint64_t per = len / ((uint64_t)(h->sm_count > 0 ? h->sm_count : 148) * per_sm + n_files);
    uint64_t s = per < floor ? floor : per;
    if (s > cap) s = cap;
    return (s + 63) & ~63ull;
}

// distinct speculative starts: about one per 128 bytes of span (measured best
// on the mixed stream for RAM and AE at 4, 8 and 16 KiB means), at most 96 for
// AE (at 16 KiB mean, 96 instead of 128 starts made a 4 GiB call 5% faster;
// RAM was slower with fewer). MAXP chains join within a chunk, so 16 starts
// cover its entries (1% faster than one per 128 bytes on the mixed stream, 15%
// on 16 MiB inputs with fewer segments).
static uint32_t pick_starts(cdc_handle h, cdc_alg alg, uint64_t span) {
    if (h->starts) return (uint32_t)h->starts;
    if (alg == CDC_MAXP) return 16u;
    uint64_t n = span / 128;
    if (n < 16) n = 16;
    const uint64_t cap = (alg == CDC_AE || alg == CDC_AE_MIN) ? 96u : (uint64_t)NL;
    if (n > cap) n = cap;
    return (uint32_t)n;
}

// segments per group of the table scan. The group kernels walk a group's
// segments one after another and the scan walks the groups one after another,
// so the latency is about gs * (compose + settle step) + (items / gs) * (scan
// step); with the scan step about a fifth of the other two, the smallest power
// of two >= sqrt(items) / 2 is near the optimum (16 for a 16 MiB input, 64 for
// 4 GiB), within GS_MIN..GS_MAX. Results do not depend on it.
static uint32_t pick_gs(uint64_t items) {
    uint32_t g = GS_MIN;
    while (g < (uint32_t)GS_MAX && 4ull * g * g < items) g *= 2;
    return g;
}

static uint64_t pick_span(cdc_handle h, cdc_params p, uint64_t seg) {
    uint64_t sp = h->span ? (uint64_t)h->span : (uint64_t)p.max / 8;
    if (sp < 32) sp = 32;
    if (sp > seg / 2) sp = seg / 2 > 32 ? seg / 2 : 32;
    return sp;
}

// summary blocks staged per segment: the segment, the room its bounds may
// move out of quiet regions (up to about twice max, see the adj_* fields),
// and max beyond its end, where its chains' last steps read
static uint32_t pick_win(cdc_params p, uint64_t seg) {
    const uint64_t mx4k = ((uint64_t)p.max + 4095) & ~4095ull;
    uint64_t blocks = (seg + 2 * mx4k + (uint64_t)p.max + 2 * 64) / 64 + 32;
    blocks = (blocks + 15) & ~15ull;
    const uint64_t cap = 24u << 10;  // bytes of shared memory per summary array
    if (blocks > cap) blocks = cap;
    return (uint32_t)blocks;
}

struct Geo {
    const uint8_t* base;
    uint64_t lo, hi, glo, ghi, nblk, nblk_pad, nsup;
};

static Geo geometry(const uint8_t* data, uint64_t len) {
    Geo g;
    uintptr_t a = (uintptr_t)data;
    g.base = (const uint8_t*)(a & ~(uintptr_t)63);
    g.lo = a & 63;
    g.hi = g.lo + len;
    g.glo = g.lo & ~15ull;
    g.ghi = (g.hi + 15) & ~15ull;
    g.nblk = (g.hi + 63) / 64;
    g.nblk_pad = (g.nblk + 15) & ~15ull;
    g.nsup = (g.hi + 4095) / 4096;
    return g;
}

// ---- candidate-graph chain stage (graph.cu) ------------------------------------

static constexpr uint64_t kGraphAutoMax = 512ull << 20;
static constexpr uint64_t kGraphAutoMaxAE = 768ull << 20;

struct GraphGeo {
    uint64_t S;
    uint32_t nseg, cap, G, nunit, win;
};

// Does the call take the candidate graph, and with which geometry? The graph
// needs every natural cut to be a candidate: min <= w + 1 for RAM and AE (the
// cut never depends on min), w >= 64 so that the block rules apply, MAXP from
// block targets. Segments of S >= max bytes (64 KiB below 64 MiB, where 128 KiB
// was up to 1.3x slower on 16 MiB of the mixed stream; see below), S / 32
// candidate slots each (a multiple of 16, at most 4096); units of about
// sqrt(segments) segments.
static bool use_graph(cdc_handle h, cdc_alg alg, cdc_params p, const Plan& pl, uint64_t len, GraphGeo* gg) {
    if (h->pipeline == 1 || h->force_bytes) return false;
    // automatic: the graph for inputs up to kGraphAutoMax (kGraphAutoMaxAE for
    // AE), where it measured as fast or faster on the mixed stream at 4 and
    // 16 KiB means; at 1 GiB the speculative segments are faster
    if (h->pipeline == 0 && len > (pl.rule == RULE_AE ? kGraphAutoMaxAE : kGraphAutoMax)) return false;
    switch (pl.rule) {
    case RULE_RAM:
    case RULE_AE:
        if (p.w < 64 || (uint64_t)p.min > (uint64_t)p.w + 1) return false;
        if (alg == CDC_AE_MIN && h->pipeline != 2) return false;
        break;
    case RULE_MAXP: break;
    default: return false;
    }
    // segment size: 64 KiB below 64 MiB, 128 KiB above (10% faster for RAM at 64
    // and 128 MiB of the mixed stream, AE unchanged); MAXP, whose targets are
    // sparse, 256 KiB from 128 MiB (5-12% faster). Larger RAM/AE segments
    // overflow their slots on text-like content.
    uint64_t S = 64u << 10;
    if (len >= (64ull << 20)) S = 128u << 10;
    if (pl.rule == RULE_MAXP && len >= (128ull << 20)) S = 256u << 10;
    if (h->graph_seg) S = (uint64_t)h->graph_seg;
    const uint64_t mx4k = ((uint64_t)p.max + 4095) & ~4095ull;
    if (S < mx4k) S = mx4k;
    if (S > (64ull << 20)) return false;
    uint64_t cap = h->graph_cap ? (uint64_t)h->graph_cap : S / 32;
    cap = (cap + 15) & ~15ull;  // slots start 16-byte aligned for vector loads
    if (cap > 4096) cap = 4096;
    if (cap < 16) cap = 16;
    const uint64_t nseg = (len + S - 1) / S;
    if (nseg == 0 || nseg * cap >= (uint64_t)GID_NONE) return false;
    gg->S = S;
    gg->nseg = (uint32_t)nseg;
    gg->cap = (uint32_t)cap;
    if (nseg <= 32) {
        gg->G = (uint32_t)nseg;
    } else {
        uint32_t G = 1;
        while ((uint64_t)G * G < nseg) G++;
        gg->G = G;
    }
    gg->nunit = (uint32_t)((nseg + gg->G - 1) / gg->G);
    // summaries staged per segment by the local kernel: the segment, max past
    // it and the windows around (multiple of 16 blocks)
    uint64_t win = (2 * S + 2ull * p.w + 256 + 63) / 64 + 32;
    win = (win + 15) & ~15ull;
    if (win > (8u << 10)) win = 8u << 10;
    gg->win = (uint32_t)win;
    return true;
}

// far landings listed per call (exits more than one segment ahead)
static size_t graph_far_cap(const GraphGeo& gg) { return (size_t)gg.nseg * 64 + 1024; }

// The candidate graph's workspace for geometry gg over summaries of nblk_pad
// blocks and nsup superblocks (the candidate kernel stages up to 1032 blocks
// past the data, so the block arrays get 2112 blocks of room).
static cdc_status graph_grow(cdc_handle h, const Plan& pl, const GraphGeo& gg, uint64_t nblk_pad, uint64_t nsup,
                             cudaStream_t st) {
    cdc_status s;
    const size_t need = nblk_pad + 2112;
    if ((s = grow(&h->smax, &h->sum_cap, need, false, st)) != CDC_OK) return s;
    if (pl.sum != SUM_MAXP && (s = grow(&h->sarg, &h->sarg_cap, need, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->ssup, &h->ssup_cap, nsup + 64, false, st)) != CDC_OK) return s;
    if (pl.rule != RULE_MAXP) {
        if ((s = grow(&h->g_spre, &h->g_spre_cap, need, false, st)) != CDC_OK) return s;
        if ((s = grow(&h->g_ssuf, &h->g_ssuf_cap, need, false, st)) != CDC_OK) return s;
    }
    const size_t slots = (size_t)gg.nseg * gg.cap;
    if ((s = grow(&h->g_cpos, &h->g_cpos_cap, slots, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_cval, &h->g_cval_cap, slots, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_ticket, &h->g_ticket_cap, 2, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_cft, &h->g_cft_cap, slots, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_csc, &h->g_csc_cap, slots, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_cex, &h->g_cex_cap, slots, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_cnum, &h->g_cnum_cap, (size_t)gg.nseg, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_sent, &h->g_sent_cap, (size_t)gg.nseg, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_soff, &h->g_soff_cap, (size_t)gg.nseg, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_uex, &h->g_uex_cap, slots, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_cfar, &h->g_cfar_cap, slots, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_far, &h->g_far_cap, graph_far_cap(gg), false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_uent, &h->g_uent_cap, (size_t)gg.nunit, false, st)) != CDC_OK) return s;
    if ((s = grow(&h->g_uoff, &h->g_uoff_cap, (size_t)gg.nunit, false, st)) != CDC_OK) return s;
    return CDC_OK;
}

static cdc_status run_graph(cdc_handle h, cdc_alg alg, cdc_params p, const Plan& pl, const Geo& g,
                            const GraphGeo& gg, uint64_t* out, uint64_t capacity, uint64_t* d_count,
                            cudaStream_t st, uint64_t ctx) {
    (void)alg;
    cdc_status s;
    if ((s = graph_grow(h, pl, gg, g.nblk_pad, g.nsup, st)) != CDC_OK) return s;
    h->launches = 0;
    const bool rec = !capturing(st);
    h->timed = false;
    cudaEvent_t* ev = h->ev;
    if (rec && h->profile && h->prof_n < cdc_handle_s::PROF_CAP) ev = h->prof_ev + 4 * h->prof_n++;
    if (h->stats) cudaMemsetAsync(h->ctrl->stats, 0, sizeof(h->ctrl->stats), st);
    if (rec) cudaEventRecord(ev[0], st);
    {
        SumLaunch a;
        memset(&a, 0, sizeof a);
        a.base = g.base;
        a.lo = g.lo; a.hi = g.hi; a.glo = g.glo; a.ghi = g.ghi;
        a.nblk = g.nblk;
        a.smax = h->smax;
        a.sarg = h->sarg;
        a.ssup = h->ssup;
        a.nsup = g.nsup;
        a.w = p.w;
        a.halo_blocks = pl.halo;
        a.timeout_ns = (uint64_t)h->timeout_ms * 1000000ull;
        a.ctrl = h->ctrl;
        if (pl.rule != RULE_MAXP) {
            a.spre = h->g_spre;
            a.ssuf = h->g_ssuf;
        }
        uint64_t tiles = summary_tiles(pl.sum, g.nblk);
        uint64_t grid = (uint64_t)h->sm_count * summary_blocks_per_sm(pl.sum, pl.halo);
        if (grid > tiles) grid = tiles;
        if (grid < 1) grid = 1;
        if (launch_summary(a, pl.sum, (int)grid, st) != cudaSuccess) return CDC_ERR_CUDA;
        h->launches++;
    }
    if (rec) cudaEventRecord(ev[1], st);
    GraphLaunch ga;
    memset(&ga, 0, sizeof ga);
    ga.base = g.base;
    ga.flo = g.lo;  // the summaries cover the context bytes too
    ga.lo = g.lo + ctx;
    ga.hi = g.hi;
    ga.smax = h->smax;
    ga.sarg = h->sarg ? h->sarg : h->smax;
    ga.ssup = h->ssup;
    ga.w = p.w; ga.mn = p.min; ga.mx = p.max;
    ga.inv = pl.inv;
    ga.S = gg.S;
    ga.nseg = gg.nseg;
    ga.cap = gg.cap;
    ga.G = gg.G;
    ga.nunit = gg.nunit;
    ga.win = gg.win;
    ga.cpos = h->g_cpos;
    ga.cval = h->g_cval;
    ga.ticket = h->g_ticket;
    ga.cnum = h->g_cnum;
    ga.cft = h->g_cft;
    ga.csc = h->g_csc;
    ga.cex = h->g_cex;
    ga.cux = h->g_uex;
    ga.cfar = h->g_cfar;
    ga.far_list = h->g_far;
    ga.far_cap = (uint32_t)graph_far_cap(gg);
    ga.uent = h->g_uent;
    ga.uoff = h->g_uoff;
    ga.sent = h->g_sent;
    ga.soff = h->g_soff;
    ga.out = out;
    ga.capacity = capacity;
    ga.d_count = d_count;
    ga.ctrl = h->ctrl;
    ga.stats = h->stats ? h->ctrl->stats : nullptr;
    ga.timeout_ns = (uint64_t)h->timeout_ms * 1000000ull;
    // running maxima inside superblocks (written by the summary kernel)
    if (pl.rule != RULE_MAXP) {
        ga.spre = h->g_spre;
        ga.ssuf = h->g_ssuf;
    }
    const uint64_t sms = (uint64_t)(h->sm_count > 0 ? h->sm_count : 148);
    auto clampg = [](uint64_t want, uint64_t lim) { return (int)(want < lim ? (want > 0 ? want : 1) : lim); };
    GraphGrids gr;
    gr.cand = clampg(gg.nseg, sms * 8);
    gr.local = clampg(gg.nseg, sms * (uint64_t)graph_local_blocks_per_sm(pl.rule, gg.cap, gg.win));
    gr.unit = clampg(gg.nunit, 65535);
    gr.emit = clampg(gg.nseg, sms * 32);
    if (launch_graph(ga, pl.rule, gr, st, &h->launches, rec ? ev[3] : nullptr) != cudaSuccess) return CDC_ERR_CUDA;
    if (rec) {
        cudaEventRecord(ev[2], st);
        h->last_ev = ev;
        h->timed = true;
    }
    h->prof_launches += h->launches;
    return CDC_OK;
}

// launch the summary and chain stages; n_files == 0 means one stream
static cdc_status run(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* data, uint64_t len,
                      const uint64_t* d_file_off, uint64_t n_files, uint64_t* out, uint64_t capacity,
                      uint64_t* bounds_index, uint64_t* d_count, cudaStream_t st, uint64_t ctx = 0) {
    cudaSetDevice(h->device);
    const Plan pl = make_plan(h, alg, p);
    // summaries cover the context bytes before data too (ctx > 0: one stream only)
    const Geo g = geometry(data - ctx, len + ctx);
    const bool batch = d_file_off != nullptr;
    const uint64_t seg = pick_seg(h, alg, p, len, batch ? n_files : 1);
    const uint64_t items = batch ? len / seg + n_files + 1 : (len + seg - 1) / seg;
    GraphGeo gg;
    // (a left context only exists for MAXP, whose targets may use it as window bytes)
    const bool graph = !batch && (ctx == 0 || pl.rule == RULE_MAXP) && use_graph(h, alg, p, pl, len, &gg);
    cdc_status s;
    h->stage = graph ? 2 : 1;
    if (graph) return run_graph(h, alg, p, pl, g, gg, out, capacity, d_count, st, ctx);
    if (pl.sum != SUM_NONE) {
        const size_t need = g.nblk_pad + 64;
        if ((s = grow(&h->smax, &h->sum_cap, need, false, st)) != CDC_OK) return s;
        if (pl.sum != SUM_MAXP && (s = grow(&h->sarg, &h->sarg_cap, need, false, st)) != CDC_OK) return s;
        if ((s = grow(&h->ssup, &h->ssup_cap, g.nsup + 64, false, st)) != CDC_OK) return s;
    }
    if ((s = grow(&h->st, &h->st_cap, items * seg_state_bytes(), true, st)) != CDC_OK) return s;
    if ((s = grow(&h->hash, &h->hash_cap, items * seg_hash_bytes(), false, st)) != CDC_OK) return s;
    if ((s = grow(&h->plog, &h->plog_cap, items * seg_log_bytes(kLogCap), false, st)) != CDC_OK) return s;
    if ((s = grow(&h->groups, &h->groups_cap, ((items + GS_MIN - 1) / GS_MIN + 1) * group_state_bytes(), false,
                  st)) != CDC_OK)
        return s;
    if (batch) {
        if ((s = grow(&h->item_off, &h->files_cap, n_files + 1, false, st)) != CDC_OK) return s;
        if ((s = grow(&h->scan_tmp, &h->scan_cap, batch_scan_tmp_elems(n_files), false, st)) != CDC_OK) return s;
        if ((s = grow(&h->item_file, &h->item_file_cap, items, false, st)) != CDC_OK) return s;
    }
    h->launches = 0;
    const uint64_t timeout_ns = (uint64_t)h->timeout_ms * 1000000ull;
    const bool rec = !capturing(st);
    h->timed = false;
    cudaEvent_t* ev = h->ev;
    if (rec && h->profile && h->prof_n < cdc_handle_s::PROF_CAP) ev = h->prof_ev + 4 * h->prof_n++;
    if (batch) {
        if (launch_batch_setup(d_file_off, n_files, seg, h->item_off, h->item_file, h->scan_tmp, h->ctrl, st,
                               &h->launches) != cudaSuccess)
            return CDC_ERR_CUDA;
    }
    if (rec) cudaEventRecord(ev[0], st);
    if (pl.sum != SUM_NONE) {
        SumLaunch a;
        memset(&a, 0, sizeof a);
        a.base = g.base;
        a.lo = g.lo; a.hi = g.hi; a.glo = g.glo; a.ghi = g.ghi;
        a.nblk = g.nblk;
        a.smax = h->smax;
        a.sarg = h->sarg;
        a.ssup = h->ssup;
        a.nsup = g.nsup;
        a.w = p.w;
        a.halo_blocks = pl.halo;
        a.timeout_ns = timeout_ns;
        a.ctrl = h->ctrl;
        uint64_t tiles = summary_tiles(pl.sum, g.nblk);
        uint64_t grid = (uint64_t)h->sm_count * summary_blocks_per_sm(pl.sum, pl.halo);
        if (grid > tiles) grid = tiles;
        if (grid < 1) grid = 1;
        if (launch_summary(a, pl.sum, (int)grid, st) != cudaSuccess) return CDC_ERR_CUDA;
    } else {
        if (launch_reset(h->ctrl, st) != cudaSuccess) return CDC_ERR_CUDA;
    }
    h->launches++;
    if (rec) cudaEventRecord(ev[1], st);
    ChainLaunch c;
    memset(&c, 0, sizeof c);
    c.base = g.base;
    c.lo = g.lo + ctx;
    c.hi = g.hi;
    c.wctx = ctx;
    c.smax = h->smax;
    c.sarg = h->sarg ? h->sarg : h->smax;
    c.ssup = h->ssup;
    c.nblk_pad = g.nblk_pad;
    c.w = p.w; c.mn = p.min; c.mx = p.max;
    c.inv = pl.inv;
    c.file_off = batch ? d_file_off : nullptr;
    c.single_len = len;
    c.n_files = batch ? n_files : 1;
    c.item_off = batch ? h->item_off : nullptr;
    c.item_file = batch ? h->item_file : nullptr;
    c.n_items = items;
    c.n_items_dev = batch ? &h->ctrl->n_items : nullptr;
    c.seg = seg;
    c.span = pick_span(h, p, seg);
    c.win = pick_win(p, seg);
    c.out = out;
    c.capacity = capacity;
    c.bounds_index = bounds_index;
    c.d_count = d_count;
    c.st = reinterpret_cast<SegState*>(h->st);
    c.hash = reinterpret_cast<unsigned long long*>(h->hash);
    c.plog = reinterpret_cast<unsigned long long*>(h->plog);
    c.logcap = kLogCap;
    c.groups = h->groups;
    c.ctrl = h->ctrl;
    c.timeout_ns = timeout_ns;
    c.hold_item = h->hold_item;
    c.stats = (int)h->stats;
    c.warp_chains = h->warp_chains ? (uint32_t)h->warp_chains : 96u;
    c.starts = pick_starts(h, alg, c.span);
    c.gs = pick_gs(items);
    if (h->stats) cudaMemsetAsync(h->ctrl->stats, 0, sizeof(h->ctrl->stats), st);
    if (pl.sum != SUM_NONE) {
        const uint64_t mx4k = ((uint64_t)p.max + 4095) & ~4095ull;
        c.quiet_run = pl.sum == SUM_MAXP ? (uint32_t)(p.max / 8192 > 1 ? p.max / 8192 : 1) : 1u;
        c.adj_before = ((mx4k / 4) + 4095) & ~4095ull;
        c.adj_after = mx4k;
        c.adj_cap = 64ull << 20;
    }
    ChainGrids gr;
    const uint64_t ngroups = (items + c.gs - 1) / c.gs;
    uint64_t gs = (uint64_t)h->sm_count * spec_blocks_per_sm(pl.rule, c.win);
    gr.spec = (int)(gs < items ? gs : items);
    gr.stitch = (int)(items < (uint64_t)h->sm_count * 8 ? items : (uint64_t)h->sm_count * 8);
    gr.groups = (int)(ngroups < (uint64_t)h->sm_count * 16 ? ngroups : (uint64_t)h->sm_count * 16);
    gr.output = (int)(items < (uint64_t)h->sm_count * 32 ? items : (uint64_t)h->sm_count * 32);
    if (gr.spec < 1) gr.spec = 1;
    if (gr.stitch < 1) gr.stitch = 1;
    if (gr.groups < 1) gr.groups = 1;
    if (gr.output < 1) gr.output = 1;
    if (launch_chain(c, pl.rule, gr, st, &h->launches, rec ? ev[3] : nullptr) != cudaSuccess) return CDC_ERR_CUDA;
    if (rec) {
        cudaEventRecord(ev[2], st);
        h->last_ev = ev;
        h->timed = true;
    }
    h->prof_launches += h->launches;
    return CDC_OK;
}

// read the control block, map device errors, clear them
static cdc_status collect(cdc_handle h, cudaStream_t st, uint64_t* total) {
    if (cudaMemcpyAsync(h->pinned_ctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return CDC_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CDC_ERR_CUDA;
    if (total) *total = h->pinned_ctrl->total;
    unsigned err = h->pinned_ctrl->err;
    if (err) {
        cudaMemsetAsync(&h->ctrl->err, 0, sizeof(unsigned), st);
        cudaStreamSynchronize(st);
        if (err & ERR_TIMEOUT) return CDC_ERR_TIMEOUT;
        return CDC_ERR_INTERNAL;
    }
    return CDC_OK;
}

extern "C" cdc_status cdc_chunk(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* data, size_t len,
                                uint64_t* out_bounds, size_t* n, cdc_stream stream) {
    if (!h || !n || !valid_params(alg, p)) return CDC_ERR_INVALID;
    if (len == 0) {
        *n = 0;
        return CDC_OK;
    }
    if (!data || !out_bounds) return CDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    cdc_status s = run(h, alg, p, data, len, nullptr, 0, out_bounds, *n, nullptr, nullptr, st);
    if (s != CDC_OK) return s;
    uint64_t total = 0;
    s = collect(h, st, &total);
    if (s != CDC_OK) return s;
    size_t cap = *n;
    *n = (size_t)total;
    return total > cap ? CDC_ERR_CAPACITY : CDC_OK;
}

cdc_status cdc::chunk_in_context(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* data, uint64_t len,
                                 uint64_t ctx, uint64_t* out, uint64_t capacity, uint64_t* d_count,
                                 cudaStream_t st) {
    return run(h, alg, p, data, len, nullptr, 0, out, capacity, nullptr, d_count, st, ctx);
}

cdc_status cdc::handle_status(cdc_handle h, cudaStream_t st) { return collect(h, st, nullptr); }

extern "C" cdc_status cdc_chunk_async(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* data, size_t len,
                                      uint64_t* out_bounds, size_t capacity, uint64_t* d_count,
                                      cdc_stream stream) {
    if (!h || !d_count || !valid_params(alg, p)) return CDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (len == 0) {
        return cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st) == cudaSuccess ? CDC_OK : CDC_ERR_CUDA;
    }
    if (!data || !out_bounds) return CDC_ERR_INVALID;
    return run(h, alg, p, data, len, nullptr, 0, out_bounds, capacity, nullptr, d_count, st);
}

extern "C" cdc_status cdc_chunk_batch(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* data,
                                      size_t data_len, const uint64_t* d_file_off, size_t n_files,
                                      uint64_t* d_bounds, uint64_t* d_bounds_index, size_t capacity,
                                      size_t* total, cdc_stream stream) {
    if (!h || !valid_params(alg, p) || !d_file_off || !d_bounds_index) return CDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_files == 0 || data_len == 0) {
        if (cudaMemsetAsync(d_bounds_index, 0, (n_files + 1) * sizeof(uint64_t), st) != cudaSuccess)
            return CDC_ERR_CUDA;
        if (total) {
            *total = 0;
            cudaStreamSynchronize(st);
        }
        return CDC_OK;
    }
    if (!data || !d_bounds || n_files > 0xFFFFFFFFull) return CDC_ERR_INVALID;
    // d_bounds_index also covers the all-empty-files case: zero it first
    if (cudaMemsetAsync(d_bounds_index, 0, (n_files + 1) * sizeof(uint64_t), st) != cudaSuccess) return CDC_ERR_CUDA;
    cdc_status s = run(h, alg, p, data, data_len, d_file_off, n_files, d_bounds, capacity, d_bounds_index,
                       nullptr, st);
    if (s != CDC_OK || !total) return s;
    uint64_t t = 0;
    s = collect(h, st, &t);
    if (s != CDC_OK) return s;
    *total = (size_t)t;
    return t > capacity ? CDC_ERR_CAPACITY : CDC_OK;
}

extern "C" cdc_status cdc_chunk_host(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* host_data, size_t len,
                                     uint64_t* host_bounds, size_t* n, cdc_stream stream) {
    if (!h || !n || !valid_params(alg, p)) return CDC_ERR_INVALID;
    if (len == 0) {
        *n = 0;
        return CDC_OK;
    }
    if (!host_data || !host_bounds) return CDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(h->device);
    cdc_status s;
    if ((s = grow(&h->host_stage, &h->host_stage_cap, len, false, st)) != CDC_OK) return s;
    size_t cap = *n;
    if ((s = grow(&h->host_out, &h->host_out_cap, cap ? cap : 1, false, st)) != CDC_OK) return s;
    if (cudaMemcpyAsync(h->host_stage, host_data, len, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return CDC_ERR_CUDA;
    s = run(h, alg, p, h->host_stage, len, nullptr, 0, h->host_out, cap, nullptr, nullptr, st);
    if (s != CDC_OK) return s;
    uint64_t total = 0;
    s = collect(h, st, &total);
    if (s != CDC_OK) return s;
    *n = (size_t)total;
    if (total > cap) return CDC_ERR_CAPACITY;
    if (cudaMemcpyAsync(host_bounds, h->host_out, total * sizeof(uint64_t), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return CDC_ERR_CUDA;
    return CDC_OK;
}

// ---- autotuner -------------------------------------------------------------------
//
// Times the chunk path on the caller's input for each (segment size,
// warp-chain threshold) pair of a small grid, twice each (CUDA events around
// the stages on `stream`), and keeps the fastest pair on the handle. Every
// setting gives identical boundaries; only the time differs.
extern "C" cdc_status cdc_autotune(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* data, size_t len,
                                   const uint64_t* d_file_off, size_t n_files, uint64_t* d_bounds,
                                   uint64_t* d_bounds_index, size_t capacity, int64_t* seg_out,
                                   int64_t* warp_chains_out, float* best_ms, cdc_stream stream) {
    if (!h || !valid_params(alg, p) || !data || !d_bounds || len == 0) return CDC_ERR_INVALID;
    const bool batch = d_file_off != nullptr;
    if (batch && (!d_bounds_index || n_files == 0 || n_files > 0xFFFFFFFFull)) return CDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (capturing(st)) return CDC_ERR_INVALID;
    cudaSetDevice(h->device);
    static const int64_t kSeg[] = {0, 128 << 10, 256 << 10, 384 << 10, 512 << 10, 1 << 20};
    static const int64_t kWarp[] = {32, 64, 96};
    static const int64_t kStarts[] = {32, 64, 128};
    const int64_t seg0 = h->seg, wc0 = h->warp_chains, ns0 = h->starts, prof0 = h->profile;
    h->profile = 0;
    float best = -1.0f;
    int64_t best_seg = seg0, best_wc = wc0, best_ns = 0;
    cdc_status err = CDC_OK;
    // segment size x warp threshold with the automatic start count, then the
    // start count on the best of those
    const int n_grid = (int)(sizeof(kSeg) / sizeof(kSeg[0]) * sizeof(kWarp) / sizeof(kWarp[0]));
    const int n_starts = (int)(sizeof(kStarts) / sizeof(kStarts[0]));
    for (int c = 0; c < n_grid + n_starts; c++) {
        {
            if (c < n_grid) {
                h->seg = kSeg[c / 3];
                h->warp_chains = kWarp[c % 3];
                h->starts = 0;
            } else {
                h->seg = best_seg;
                h->warp_chains = best_wc;
                h->starts = kStarts[c - n_grid];
            }
            const int64_t sg = h->seg, wc = h->warp_chains, ns = h->starts;
            float t = -1.0f;
            for (int rep = 0; rep < 2 && err == CDC_OK; rep++) {
                if (batch && cudaMemsetAsync(d_bounds_index, 0, (n_files + 1) * sizeof(uint64_t), st) != cudaSuccess) {
                    err = CDC_ERR_CUDA;
                    break;
                }
                cdc_status s = run(h, alg, p, data, len, d_file_off, batch ? n_files : 0, d_bounds, capacity,
                                   batch ? d_bounds_index : nullptr, nullptr, st);
                uint64_t total = 0;
                if (s == CDC_OK) s = collect(h, st, &total);
                if (s == CDC_OK && total > capacity) s = CDC_ERR_CAPACITY;
                if (s != CDC_OK) {
                    err = s;
                    break;
                }
                float a = 0, b = 0;
                cudaEventElapsedTime(&a, h->ev[0], h->ev[1]);
                cudaEventElapsedTime(&b, h->ev[1], h->ev[2]);
                if (t < 0 || a + b < t) t = a + b;
            }
            if (err != CDC_OK) break;
            if (best < 0 || t < best) {
                best = t;
                best_seg = sg;
                best_wc = wc;
                best_ns = ns;
            }
        }
        if (err != CDC_OK) break;
    }
    h->profile = prof0;
    h->timed = false;
    if (err != CDC_OK) {
        h->seg = seg0;
        h->warp_chains = wc0;
        h->starts = ns0;
        return err;
    }
    h->seg = best_seg;
    h->warp_chains = best_wc;
    h->starts = best_ns;
    if (seg_out) *seg_out = best_seg;
    if (warp_chains_out) *warp_chains_out = best_wc;
    if (best_ms) *best_ms = best;
    return CDC_OK;
}

extern "C" cdc_status cdc_reserve(cdc_handle h, cdc_alg alg, cdc_params p, size_t len, size_t n_files) {
    if (!h || !valid_params(alg, p)) return CDC_ERR_INVALID;
    cudaSetDevice(h->device);
    const Plan pl = make_plan(h, alg, p);
    const uint64_t nblk_pad = ((len + 64 + 63) / 64 + 15) & ~15ull;
    const uint64_t seg = pick_seg(h, alg, p, len, n_files ? n_files : 1);
    const uint64_t items = len / seg + n_files + 2;
    cdc_status s;
    if (pl.sum != SUM_NONE) {
        if ((s = grow(&h->smax, &h->sum_cap, nblk_pad + 64, false, 0)) != CDC_OK) return s;
        if (pl.sum != SUM_MAXP && (s = grow(&h->sarg, &h->sarg_cap, nblk_pad + 64, false, 0)) != CDC_OK) return s;
    }
    if (pl.sum != SUM_NONE && (s = grow(&h->ssup, &h->ssup_cap, len / 4096 + 66, false, 0)) != CDC_OK) return s;
    if ((s = grow(&h->st, &h->st_cap, items * seg_state_bytes(), true, 0)) != CDC_OK) return s;
    if ((s = grow(&h->hash, &h->hash_cap, items * seg_hash_bytes(), false, 0)) != CDC_OK) return s;
    if ((s = grow(&h->plog, &h->plog_cap, items * seg_log_bytes(kLogCap), false, 0)) != CDC_OK) return s;
    if ((s = grow(&h->groups, &h->groups_cap, ((items + GS_MIN - 1) / GS_MIN + 1) * group_state_bytes(), false,
                  0)) != CDC_OK)
        return s;
    if (n_files) {
        if ((s = grow(&h->item_off, &h->files_cap, n_files + 1, false, 0)) != CDC_OK) return s;
        if ((s = grow(&h->scan_tmp, &h->scan_cap, batch_scan_tmp_elems(n_files), false, 0)) != CDC_OK) return s;
        if ((s = grow(&h->item_file, &h->item_file_cap, items, false, 0)) != CDC_OK) return s;
    } else {
        // a single stream may take the candidate graph (with the handle's options as they are now)
        GraphGeo gg;
        if (len && use_graph(h, alg, p, pl, len, &gg) &&
            (s = graph_grow(h, pl, gg, nblk_pad, len / 4096 + 2, 0)) != CDC_OK)
            return s;
    }
    return CDC_OK;
}

extern "C" cdc_status cdc_sync_status(cdc_handle h, cdc_stream stream) {
    if (!h) return CDC_ERR_INVALID;
    return collect(h, (cudaStream_t)stream, nullptr);
}

extern "C" cdc_status cdc_last_timing(cdc_handle h, float* summary_ms, float* chain_ms) {
    if (!h || !h->timed || !h->last_ev) return CDC_ERR_INVALID;
    cudaEvent_t* ev = h->last_ev;
    if (cudaEventSynchronize(ev[2]) != cudaSuccess) return CDC_ERR_CUDA;
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b, ev[1], ev[2]);
    if (summary_ms) *summary_ms = a;
    if (chain_ms) *chain_ms = b;
    return CDC_OK;
}

extern "C" cdc_status cdc_last_launches(cdc_handle h, int* launches) {
    if (!h || !launches) return CDC_ERR_INVALID;
    *launches = h->launches;
    return CDC_OK;
}

extern "C" cdc_status cdc_last_stage(cdc_handle h, int* stage) {
    if (!h || !stage) return CDC_ERR_INVALID;
    *stage = h->stage;
    return CDC_OK;
}

extern "C" cdc_status cdc_profile_collect(cdc_handle h, int* calls, double* summary_ms, double* chain_ms,
                                          double* spec_ms, int64_t* launches) {
    if (!h) return CDC_ERR_INVALID;
    double a = 0, b = 0, c = 0;
    for (int i = 0; i < h->prof_n; i++) {
        cudaEvent_t* ev = h->prof_ev + 4 * i;
        if (cudaEventSynchronize(ev[2]) != cudaSuccess) return CDC_ERR_CUDA;
        float x = 0, y = 0, z = 0;
        cudaEventElapsedTime(&x, ev[0], ev[1]);
        cudaEventElapsedTime(&y, ev[1], ev[2]);
        cudaEventElapsedTime(&z, ev[1], ev[3]);
        a += x;
        b += y;
        c += z;
    }
    if (calls) *calls = h->prof_n;
    if (summary_ms) *summary_ms = a;
    if (chain_ms) *chain_ms = b;
    if (spec_ms) *spec_ms = c;
    if (launches) *launches = h->prof_launches;
    h->prof_n = 0;
    h->prof_launches = 0;
    h->last_ev = nullptr;
    h->timed = false;
    return CDC_OK;
}

extern "C" cdc_status cdc_stats(cdc_handle h, uint64_t* out, int n, cdc_stream stream) {
    if (!h || !out || n < 0) return CDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(h->pinned_ctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return CDC_ERR_CUDA;
    for (int i = 0; i < n && i < STAT_N; i++) out[i] = h->pinned_ctrl->stats[i];
    return CDC_OK;
}

// ---- cdc_chunk_static: the chunk path on one fixed scratch array ----------------
//
// Same plan, kernels and launch order as run() for a single stream, but every
// workspace pointer points into g_fixed_scratch, so nothing is allocated.
// Layout (byte offsets, each part 256-byte aligned):
//   control block | smax | sarg | ssup | segment states | group states | segment hashes | step logs

namespace {
constexpr uint64_t round256(uint64_t x) { return (x + 255) & ~255ull; }
constexpr uint64_t kFixMaxLen = CDC_STATIC_MAX_LEN;
constexpr uint64_t kFixMinSeg = 32u << 10;  // pick_seg() never picks less
// data may start up to 63 bytes into its 64-byte block
constexpr uint64_t kFixBlocks = ((kFixMaxLen + 63 + 63) / 64 + 15) & ~15ull;
constexpr uint64_t kFixSumBytes = round256(kFixBlocks + 64);
constexpr uint64_t kFixSupBytes = round256((kFixMaxLen + 63 + 4095) / 4096 + 64);
constexpr uint64_t kFixItems = kFixMaxLen / kFixMinSeg + 1;
constexpr uint64_t kFixSegSlot = 4096;    // >= sizeof(SegState), checked at set-up
constexpr uint64_t kFixGroupSlot = 2048;  // >= sizeof(GroupState), checked at set-up
constexpr uint64_t kFixHashSlot = 16384;  // >= a segment's position hash, checked at set-up
constexpr uint32_t kFixLogCap = 1024;     // speculation steps logged per segment
constexpr uint64_t kFixLogSlot = 20480;   // >= a segment's step logs, checked at set-up
constexpr uint64_t kFixGroups = kFixItems / GS_MIN + 2;
constexpr uint64_t kFixCtrlBytes = 512;
constexpr uint64_t kFixOffSmax = kFixCtrlBytes;
constexpr uint64_t kFixOffSarg = kFixOffSmax + kFixSumBytes;
constexpr uint64_t kFixOffSup = kFixOffSarg + kFixSumBytes;
constexpr uint64_t kFixOffSt = kFixOffSup + kFixSupBytes;
constexpr uint64_t kFixOffGroups = kFixOffSt + kFixItems * kFixSegSlot;
constexpr uint64_t kFixOffHash = kFixOffGroups + kFixGroups * kFixGroupSlot;
constexpr uint64_t kFixOffLog = kFixOffHash + kFixItems * kFixHashSlot;
constexpr uint64_t kFixTotal = kFixOffLog + kFixItems * kFixLogSlot;
static_assert(kFixTotal == CDC_STATIC_SCRATCH_BYTES, "scratch layout and header disagree");
static_assert(sizeof(Ctrl) <= kFixCtrlBytes, "control block does not fit");
constexpr int kFixMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_fixed_scratch[kFixTotal];

static std::mutex g_fixed_mu;
static uint8_t* g_fixed_ptr[kFixMaxDevices];  // device address of the scratch, per device

// Device address of the scratch on `dev` (the current device). The first call
// per device looks it up and zeroes the control block (its epoch counter) and
// the segment states (their ready flags); later calls only read the cache.
static cdc_status fixed_scratch(int dev, cudaStream_t st, uint8_t** out) {
    if (dev < 0 || dev >= kFixMaxDevices) return CDC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_fixed_mu);
    if (!g_fixed_ptr[dev]) {
        if (seg_state_bytes() > kFixSegSlot || group_state_bytes() > kFixGroupSlot ||
            seg_hash_bytes() > kFixHashSlot || seg_log_bytes(kFixLogCap) > kFixLogSlot)
            return CDC_ERR_INTERNAL;
        uint8_t* p = nullptr;
        if (cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_fixed_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CDC_ERR_CUDA;
        }
        if (cudaMemsetAsync(p, 0, kFixCtrlBytes, st) != cudaSuccess ||
            cudaMemsetAsync(p + kFixOffSt, 0, kFixItems * kFixSegSlot, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return CDC_ERR_CUDA;
        g_fixed_ptr[dev] = p;
    }
    *out = g_fixed_ptr[dev];
    return CDC_OK;
}

// true when p is memory of device `dev` or managed memory
static bool device_memory_of(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

extern "C" cdc_status cdc_chunk_static(cdc_alg alg, cdc_params p, const uint8_t* data, size_t len,
                                       uint64_t* out_bounds, size_t* n, cdc_stream stream) {
    if (!n || !valid_params(alg, p)) return CDC_ERR_INVALID;
    if (len == 0) {
        *n = 0;
        return CDC_OK;
    }
    if (!data || !out_bounds || len > kFixMaxLen) return CDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CDC_ERR_CUDA;
    if (!device_memory_of(data, dev) || !device_memory_of(out_bounds, dev)) return CDC_ERR_INVALID;
    uint8_t* scr = nullptr;
    cdc_status s = fixed_scratch(dev, st, &scr);
    if (s != CDC_OK) return s;
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(scr);

    // the plan and geometry a default handle would pick (fields are only read)
    cdc_handle_s cfg;
    cfg.device = dev;
    cudaDeviceGetAttribute(&cfg.sm_count, cudaDevAttrMultiProcessorCount, dev);
    const Plan pl = make_plan(&cfg, alg, p);
    const Geo g = geometry(data, len);
    const uint64_t seg = pick_seg(&cfg, alg, p, len, 1);
    const uint64_t items = (len + seg - 1) / seg;
    if (items > kFixItems || g.nblk_pad + 64 > kFixSumBytes || g.nsup + 64 > kFixSupBytes) return CDC_ERR_INTERNAL;
    const uint64_t timeout_ns = (uint64_t)cfg.timeout_ms * 1000000ull;

    if (cudaMemsetAsync(&ctrl->err, 0, sizeof(unsigned int), st) != cudaSuccess) return CDC_ERR_CUDA;
    int launches = 0;
    if (pl.sum != SUM_NONE) {
        SumLaunch a;
        memset(&a, 0, sizeof a);
        a.base = g.base;
        a.lo = g.lo; a.hi = g.hi; a.glo = g.glo; a.ghi = g.ghi;
        a.nblk = g.nblk;
        a.smax = scr + kFixOffSmax;
        a.sarg = pl.sum != SUM_MAXP ? scr + kFixOffSarg : nullptr;
        a.ssup = scr + kFixOffSup;
        a.nsup = g.nsup;
        a.w = p.w;
        a.halo_blocks = pl.halo;
        a.timeout_ns = timeout_ns;
        a.ctrl = ctrl;
        uint64_t tiles = summary_tiles(pl.sum, g.nblk);
        uint64_t grid = (uint64_t)cfg.sm_count * summary_blocks_per_sm(pl.sum, pl.halo);
        if (grid > tiles) grid = tiles;
        if (grid < 1) grid = 1;
        if (launch_summary(a, pl.sum, (int)grid, st) != cudaSuccess) return CDC_ERR_CUDA;
    } else {
        if (launch_reset(ctrl, st) != cudaSuccess) return CDC_ERR_CUDA;
    }
    ChainLaunch c;
    memset(&c, 0, sizeof c);
    c.base = g.base;
    c.lo = g.lo;
    c.hi = g.hi;
    c.smax = scr + kFixOffSmax;
    c.sarg = pl.sum != SUM_MAXP ? scr + kFixOffSarg : scr + kFixOffSmax;
    c.ssup = scr + kFixOffSup;
    c.nblk_pad = g.nblk_pad;
    c.w = p.w; c.mn = p.min; c.mx = p.max;
    c.inv = pl.inv;
    c.file_off = nullptr;
    c.single_len = len;
    c.n_files = 1;
    c.n_items = items;
    c.seg = seg;
    c.span = pick_span(&cfg, p, seg);
    c.starts = pick_starts(&cfg, alg, c.span);
    c.win = pick_win(p, seg);
    c.out = out_bounds;
    c.capacity = *n;
    c.st = reinterpret_cast<SegState*>(scr + kFixOffSt);
    c.hash = reinterpret_cast<unsigned long long*>(scr + kFixOffHash);
    c.plog = reinterpret_cast<unsigned long long*>(scr + kFixOffLog);
    c.logcap = kFixLogCap;
    c.groups = scr + kFixOffGroups;
    c.ctrl = ctrl;
    c.timeout_ns = timeout_ns;
    c.hold_item = -1;
    c.warp_chains = 96u;
    c.gs = pick_gs(items);
    if (pl.sum != SUM_NONE) {
        const uint64_t mx4k = ((uint64_t)p.max + 4095) & ~4095ull;
        c.quiet_run = pl.sum == SUM_MAXP ? (uint32_t)(p.max / 8192 > 1 ? p.max / 8192 : 1) : 1u;
        c.adj_before = ((mx4k / 4) + 4095) & ~4095ull;
        c.adj_after = mx4k;
        c.adj_cap = 64ull << 20;
    }
    ChainGrids gr;
    const uint64_t ngroups = (items + c.gs - 1) / c.gs;
    const uint64_t gs = (uint64_t)cfg.sm_count * spec_blocks_per_sm(pl.rule, c.win);
    gr.spec = (int)(gs < items ? gs : items);
    gr.stitch = (int)(items < (uint64_t)cfg.sm_count * 8 ? items : (uint64_t)cfg.sm_count * 8);
    gr.groups = (int)(ngroups < (uint64_t)cfg.sm_count * 16 ? ngroups : (uint64_t)cfg.sm_count * 16);
    gr.output = (int)(items < (uint64_t)cfg.sm_count * 32 ? items : (uint64_t)cfg.sm_count * 32);
    if (gr.spec < 1) gr.spec = 1;
    if (gr.stitch < 1) gr.stitch = 1;
    if (gr.groups < 1) gr.groups = 1;
    if (gr.output < 1) gr.output = 1;
    if (launch_chain(c, pl.rule, gr, st, &launches) != cudaSuccess) return CDC_ERR_CUDA;

    // count and error word back to pageable host memory (no staging buffer of ours)
    uint64_t total = 0;
    unsigned int err = 0;
    if (cudaMemcpyAsync(&total, &ctrl->total, sizeof total, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&err, &ctrl->err, sizeof err, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return CDC_ERR_CUDA;
    if (err) {
        cudaMemsetAsync(&ctrl->err, 0, sizeof(unsigned int), st);
        cudaStreamSynchronize(st);
        return (err & ERR_TIMEOUT) ? CDC_ERR_TIMEOUT : CDC_ERR_INTERNAL;
    }
    const size_t cap = *n;
    *n = (size_t)total;
    return total > cap ? CDC_ERR_CAPACITY : CDC_OK;
}
