// cdc_device.cuh -- device-side structures and PTX helpers shared by the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "chain_logic.cuh"

namespace cdc {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr int KF = 8;  // positions per chain kept for stitching

// Control block of a handle (device memory, one per handle).
struct Ctrl {
    unsigned long long ticket;   // next segment to take (dynamic, launch order)
    unsigned long long total;    // number of boundaries (written by the last segment)
    unsigned long long n_items;  // segments of a batch (written by the batch set-up)
    unsigned long long err_info; // first failing item / position, for diagnostics
    unsigned int epoch;          // launch number; a flag is set when it equals this
    unsigned int err;            // sticky error bits, cleared by the host
    unsigned int stats_on;       // 1: kernels accumulate the counters below
    unsigned int pad[5];
    unsigned long long stats[25];  // see STAT_* (reset by the host)
};
enum : int {
    STAT_SEGMENTS = 0,      // non-empty segments speculated
    STAT_THREAD_STEPS = 1,  // chain steps taken by single threads
    STAT_WARP_STEPS = 2,    // chain steps taken by whole warps (speculation)
    STAT_MERGES = 3,        // speculative chains stopped on another chain's position
    STAT_STITCH_WALKS = 4,  // distinct predecessor exits followed
    STAT_STITCH_STEPS = 5,
    STAT_UNKNOWN = 6,       // table entries no chain covered
    STAT_HASH_FULL = 7,     // segments whose position hash filled up
    STAT_SCAN_FOLLOWS = 8,  // segments followed in the scan / settle fallback
    STAT_OUT_STEPS = 9,     // steps of the output walks
    STAT_EMPTY = 10,        // empty segments
    STAT_SURVIVORS = 11,    // chains handed to whole warps
    STAT_CYC_SETUP = 12,    // cycles (summed over CTAs): bounds + staging
    STAT_CYC_THREADS = 13,  //   per-thread speculation rounds
    STAT_CYC_WARPS = 14,    //   whole-warp survivors + merge resolution
    STAT_CYC_STITCH = 15,   //   waiting for the predecessor + stitching
    STAT_ROUNDS = 16,       // per-thread rounds (summed over segments)
    STAT_CYC_ROUNDS = 17,   //   their cycles (part of STAT_CYC_THREADS)
    STAT_CYC_SURV = 18,     // cycles of the one-warp-per-chain phase (part of STAT_CYC_THREADS)
    STAT_STITCH_LONG = 19,  // stitch walks of more than 64 steps
    STAT_STITCH_MAXW = 20,  // (steps << 32) | segment of the longest stitch walk
    STAT_OUT_PASSES = 21,   // passes of the output kernel over a step log
    STAT_OUT_RECS = 22,     // step-log records the output kernel replayed
    STAT_CYC_OUTPUT = 23,   // cycles of the output kernel, summed over segments
    STAT_CYC_OUT_STEPS = 24, //   of which in its own chain steps
    STAT_N = 25
};
enum : unsigned int { ERR_TIMEOUT = 1u, ERR_INTERNAL = 2u };

// Speculation geometry of the chain stage.
constexpr int NW = 4;            // warps per segment
constexpr int NL = 32 * NW;      // speculative chains per segment
// Segments per group in the table scan: chosen per call between these bounds
// (group walks are serial within a group, the scan is serial across groups)
constexpr int GS_MIN = 8;
constexpr int GS_MAX = 128;

#if defined(__CUDACC__)

__device__ __forceinline__ uint32_t ld_acquire(const unsigned int* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned int* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_volatile(const unsigned int* p) {
    return *reinterpret_cast<const volatile unsigned int*>(p);
}
__device__ __forceinline__ uint64_t gtimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- shared-memory barriers and 1-D bulk copies (TMA, no tensor map) -------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait on an mbarrier phase. Returns false when `limit_ns` passes.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = gtimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (gtimer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

#endif  // __CUDACC__

}  // namespace cdc
