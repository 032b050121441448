// cdc_launch.h -- launch descriptors shared by the host API and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cdc {

struct Ctrl;
struct SegState;

enum SumKind { SUM_NONE = 0, SUM_MAX = 1, SUM_MAX_INV = 2, SUM_MAXP = 3 };

// Stage 1 (block summaries). Positions are offsets from `base` (64-byte
// aligned); the data is [lo, hi); reads stay inside [glo, ghi) (16-byte granules).
struct SumLaunch {
    const uint8_t* base;
    uint64_t lo, hi, glo, ghi;
    uint64_t nblk;          // blocks of 64 bytes covering [0, hi)
    uint8_t* smax;          // per block: max (RAM/AE) or target offset / 0xFF (MAXP)
    uint8_t* sarg;          // per block: first position of the max (RAM/AE)
    uint8_t* ssup;          // per 4 KiB superblock: max byte (RAM/AE) or target count (MAXP)
    uint8_t* spre;          // RAM/AE, may be null: per block, the maximum of its superblock's blocks up to it
    uint8_t* ssuf;          //   and from it to the superblock's end
    uint64_t nsup;          // superblocks covering [0, hi)
    uint32_t w;             // MAXP window
    uint32_t halo_blocks;   // MAXP: blocks staged on each side of a tile
    uint64_t timeout_ns;
    Ctrl* ctrl;
};

// Stage 2 (speculative chains, stitching, resolution, output).
struct ChainLaunch {
    const uint8_t* base;
    uint64_t lo, hi;
    const uint8_t* smax;
    const uint8_t* sarg;
    const uint8_t* ssup;     // 4 KiB superblock summaries (quiet-region detection)
    uint64_t nblk_pad;       // summary arrays hold at least nblk_pad + 64 bytes
    uint32_t w, mn, mx;
    uint32_t inv;            // 0xFFFFFFFF for AE-Min (complemented bytes)
    // files: either one stream [0, single_len) or n_files files given by
    // file_off (logical offsets), with item_off / item_file from the batch set-up
    const uint64_t* file_off;
    uint64_t single_len;
    // one stream only: bytes before its start that belong to the same data
    // (a resumed stream); MAXP windows may reach into them, chains start at lo
    uint64_t wctx;
    uint64_t n_files;
    const uint64_t* item_off;
    const uint32_t* item_file;
    uint64_t n_items;        // used when n_items_dev is NULL
    const unsigned long long* n_items_dev;
    uint64_t seg, span;
    uint32_t win;            // summary blocks staged per segment (multiple of 16)
    // segment bounds move out of quiet regions: runs of quiet_run quiet
    // superblocks (0 = never move) within [y - adj_before, y + adj_after);
    // a bound moves at most adj_cap bytes
    uint32_t quiet_run;
    uint64_t adj_before, adj_after, adj_cap;
    // outputs
    uint64_t* out;
    uint64_t capacity;
    uint64_t* bounds_index;  // batch: n_files + 1 entries, else NULL
    uint64_t* d_count;       // receives the total, may be NULL
    // workspace
    SegState* st;
    unsigned long long* hash;  // per segment: its position hash (seg_hash_bytes())
    unsigned long long* plog;  // per segment: its step logs (seg_log_bytes(logcap))
    uint32_t logcap;           // speculation-log records per segment
    void* groups;            // GroupState per group of gs segments
    Ctrl* ctrl;
    uint64_t timeout_ns;
    int64_t hold_item;
    int stats;               // accumulate Ctrl::stats
    uint32_t warp_chains;    // per-thread speculation rounds run while more chains than this are alive
    uint32_t starts;         // distinct speculative starts per segment (threads beyond repeat them)
    uint32_t gs;             // segments per group of the table scan (GS_MIN..GS_MAX)
};

// Memo of per-device launch properties: fn(arg) runs once per (device, key, arg).
int launch_memo(int key, uint32_t arg, int (*fn)(uint32_t));

// Let `kernel` take any dynamic shared memory the current device allows
// (launches still request only what they use). Returns a cudaError_t.
template <typename K>
int allow_max_smem(K kernel) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return (int)e;
}

int summary_max_smem();
int summary_maxp_smem(uint32_t halo_blocks);
uint32_t maxp_halo_blocks(uint32_t w);
int summary_blocks_per_sm(int kind, uint32_t halo_blocks);
uint64_t summary_tiles(int kind, uint64_t nblk);
cudaError_t launch_summary(const SumLaunch& a, int kind, int grid, cudaStream_t st);
cudaError_t launch_reset(Ctrl* ctrl, cudaStream_t st);

struct ChainGrids {
    int spec, stitch, groups, output;
};
int chain_smem(int rule, uint32_t win);
int spec_blocks_per_sm(int rule, uint32_t win);
size_t seg_state_bytes();
size_t seg_hash_bytes();
size_t seg_log_bytes(uint32_t logcap);
// speculation steps a handle logs per segment (a segment with more is output by stepping)
constexpr uint32_t HANDLE_LOG_CAP = 2048;
size_t group_state_bytes();
// ev_spec (may be null) is recorded on `st` right after the speculation kernel
cudaError_t launch_chain(const ChainLaunch& a, int rule, const ChainGrids& g, cudaStream_t st, int* launches,
                         cudaEvent_t ev_spec = nullptr);

// ---- the candidate-graph chain stage (graph.cu) -------------------------------
//
// One stream [lo, hi) cut into nseg segments of S bytes (S >= max). Candidate
// ids are seg * cap + index of the candidate in its segment's slot. Special ids:
constexpr uint32_t GID_END = 0xFFFFFFFFu;   // the end of the data
constexpr uint32_t GID_SLOW = 0xFFFFFFFEu;  // a candidate beyond its segment's slot
constexpr uint32_t GID_NONE = 0xFFFFFFFDu;  // no entry

struct GraphLaunch {
    const uint8_t* base;
    uint64_t lo, hi;         // physical positions of the data (offsets from base)
    uint64_t flo;            // where the stream's bytes begin (<= lo: MAXP's left context before lo)
    uint64_t timeout_ns;     // limit of every wait (the chase kernels' staging copies)
    const uint8_t* smax;
    const uint8_t* sarg;
    const uint8_t* ssup;
    uint32_t w, mn, mx;
    uint32_t inv;
    uint64_t S;              // segment bytes (multiple of 64, >= mx)
    uint32_t nseg;
    uint32_t cap;            // candidate slots per segment
    uint32_t G;              // segments per unit of the unit tables
    uint32_t nunit;          // ceil(nseg / G); 1 = no unit tables
    uint32_t win;            // block maxima staged per segment by the local kernel
    // RAM / AE: running maxima inside superblocks (the summary kernel's spre, ssuf)
    const uint8_t* spre;     // null: none (MAXP)
    const uint8_t* ssuf;
    uint32_t* cpos;          // [nseg * cap] candidate position - segment start
    uint8_t* cval;           // [nseg * cap] its source byte (RAM: the cut byte; AE: the target)
    uint32_t* cnum;          // [nseg] candidates of the segment (may exceed cap)
    uint32_t* cft;           // [nseg * cap] id of F(candidate)
    uint32_t* csc;           // [nseg * cap] chunk ends from the candidate to F(candidate)
    unsigned long long* cex; // [nseg * cap] (ends << 32) | id of the first candidate past the segment
    unsigned long long* cux; // [nseg * cap] the same past the unit: for the unit's first segment and far landings
    uint8_t* cfar;           // [nseg * cap] 1: cux holds the candidate's unit exit (a far landing)
    uint32_t* far_list;      // far landings (F targets past the next segment), in no order
    uint32_t far_cap;
    uint32_t* uent;          // [nunit] id of the true chain's first candidate in the unit, or GID_NONE
    uint64_t* uoff;          // [nunit] boundaries before it
    uint32_t* sent;          // [nseg] id of the true chain's entry in the segment, or GID_NONE
    uint64_t* soff;          // [nseg] boundaries before it
    uint64_t* out;
    uint64_t capacity;
    uint64_t* d_count;
    Ctrl* ctrl;
    unsigned long long* ticket;  // [2]: work counter of the local kernel, far landings listed (zeroed by k_gcand)
    unsigned long long* stats;   // counters GST_* (testing only), or null
};
// counters of the candidate graph (Ctrl::stats when CDC_OPT_STATS is on)
enum : int {
    GST_SEGMENTS = 0,      // segments the local kernel processed
    GST_CANDS = 1,         // candidates
    GST_GENERIC = 2,       // F by stepping the chain (the list could not decide)
    GST_CYC_STAGE = 3,     // local kernel cycles, summed over segments: staging lists, maxima, table
    GST_CYC_F = 4,         //   F of the segment's candidates
    GST_CYC_JUMP = 5,      //   pointer jumping
    GST_ROUNDS = 6,        // jumping rounds, summed
    GST_MAX_SEG = 7,       // the longest segment (cycles)
    GST_CYC_GENERIC = 8,   // cycles of the stepped F, summed over candidates
    GST_MAX_GENERIC = 9,   // the longest stepped F (cycles)
    GST_CC_STAGE = 10,     // candidate kernel cycles, summed over chunks: staging
    GST_CC_LIST = 11,      //   listing the blocks that can hold a candidate
    GST_CC_BLOCKS = 12,    //   testing the listed blocks' bytes
    GST_CC_WRITE = 13,     //   writing the candidates
    GST_CC_LISTED = 14,    // blocks listed
    GST_MAX_STAGE = 15,    // local kernel, the longest segment of each phase (cycles): staging
    GST_MAX_F = 16,        //   F
    GST_MAX_JUMP = 17,     //   pointer jumping
    GST_MAX_SEG_AT = 18,   // (cycles << 24) | segment of the longest local segment
    GST_CC_MAX = 19        // candidate kernel: the longest chunk (cycles)
};

struct GraphGrids {
    int cand, local, unit, emit;
};
// dynamic shared memory of the local kernel (cap slots, win staged summary blocks)
int graph_local_smem(int rule, uint32_t cap, uint32_t win);
int graph_local_blocks_per_sm(int rule, uint32_t cap, uint32_t win);
cudaError_t launch_graph(const GraphLaunch& a, int rule, const GraphGrids& g, cudaStream_t st, int* launches,
                         cudaEvent_t ev_mid = nullptr);

// batch set-up: item_off (n_files + 1), item_file, ctrl->n_items
cudaError_t launch_batch_setup(const uint64_t* file_off, uint64_t n_files, uint64_t seg, uint64_t* item_off,
                               uint32_t* item_file, uint64_t* scan_tmp, Ctrl* ctrl, cudaStream_t st,
                               int* launches);
uint64_t batch_scan_tmp_elems(uint64_t n_files);

}  // namespace cdc

#include "../../include/cdc.h"

namespace cdc {

// cdc_chunk_async of [data, data + len) whose `ctx` bytes before `data` belong
// to the same stream: the chain starts at data, MAXP windows may read the
// context. The count (boundaries are offsets from data) goes to *d_count.
cdc_status chunk_in_context(cdc_handle h, cdc_alg alg, cdc_params p, const uint8_t* data, uint64_t len,
                            uint64_t ctx, uint64_t* out, uint64_t capacity, uint64_t* d_count, cudaStream_t st);
// Synchronise st and report (and clear) the handle's device-side errors.
cdc_status handle_status(cdc_handle h, cudaStream_t st);

}  // namespace cdc
