// batch.cu -- set-up for chunking many files in one launch.
//
// Every file is cut into segments of `seg` bytes; segments are numbered file
// after file, so that the chain stage can take them in order and look back
// within a file. This computes item_off[f] (first segment of file f, an
// exclusive prefix sum of the per-file segment counts), item_file[i] (file of
// segment i) and the total in ctrl->n_items, all on the device.
#include "cdc_device.cuh"
#include "cdc_launch.h"

namespace cdc {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER_THREAD = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

__device__ __forceinline__ uint64_t seg_count(const uint64_t* off, uint64_t f, uint64_t seg) {
    uint64_t len = off[f + 1] - off[f];
    return (len + seg - 1) / seg;
}

// block-wide exclusive scan of 64-bit values (one per thread)
__device__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* total) {
    __shared__ uint64_t warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t o = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += o;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint64_t s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t o = __shfl_up_sync(FULL, s, d);
            if (lane >= d) s += o;
        }
        warp_sums[lane] = s;  // inclusive
    }
    __syncthreads();
    uint64_t before = wid ? warp_sums[wid - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

// pass 1: per-tile exclusive scan of segment counts; tile sums to tmp
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const uint64_t* off, uint64_t n, uint64_t seg,
                                                             uint64_t* item_off, uint64_t* tile_sum) {
    const uint64_t t0 = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_PER_THREAD;
    uint64_t v[SCAN_PER_THREAD], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; k++) {
        v[k] = t0 + k < n ? seg_count(off, t0 + k, seg) : 0;
        s += v[k];
    }
    uint64_t tot;
    uint64_t ex = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; k++) {
        if (t0 + k < n) item_off[t0 + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// pass 2: exclusive scan of the tile sums (one CTA, any count)
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_sums(uint64_t* tile_sum, uint64_t ntiles, uint64_t* item_off,
                                                            uint64_t n, Ctrl* ctrl) {
    uint64_t carry = 0;
    for (uint64_t b = 0; b < ntiles; b += SCAN_THREADS) {
        uint64_t i = b + threadIdx.x;
        uint64_t v = i < ntiles ? tile_sum[i] : 0, tot;
        uint64_t ex = block_exclusive_scan(v, &tot);
        if (i < ntiles) tile_sum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        item_off[n] = carry;
        ctrl->n_items = carry;
    }
}

// pass 3: add tile offsets; write the file of every segment
__global__ void k_scan_finish(uint64_t* item_off, const uint64_t* tile_sum, const uint64_t* off, uint64_t n,
                              uint64_t seg, uint32_t* item_file) {
    const uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    uint64_t io = item_off[f] + tile_sum[f / SCAN_TILE];
    item_off[f] = io;
    uint64_t c = seg_count(off, f, seg);
    for (uint64_t k = 0; k < c; k++) item_file[io + k] = (uint32_t)f;
}

uint64_t batch_scan_tmp_elems(uint64_t n_files) { return (n_files + SCAN_TILE - 1) / SCAN_TILE + 1; }

cudaError_t launch_batch_setup(const uint64_t* file_off, uint64_t n_files, uint64_t seg, uint64_t* item_off,
                               uint32_t* item_file, uint64_t* scan_tmp, Ctrl* ctrl, cudaStream_t st,
                               int* launches) {
    const uint64_t ntiles = (n_files + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_tiles<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(file_off, n_files, seg, item_off, scan_tmp);
    k_scan_sums<<<1, SCAN_THREADS, 0, st>>>(scan_tmp, ntiles, item_off, n_files, ctrl);
    k_scan_finish<<<(unsigned)((n_files + 255) / 256), 256, 0, st>>>(item_off, scan_tmp, file_off, n_files, seg,
                                                                     item_file);
    *launches += 3;
    return cudaGetLastError();
}

}  // namespace cdc
