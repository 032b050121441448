// feed.cu -- resumable chunking of a stream that arrives in pieces
// (include/cdc.h, cdc_feed_*).
//
// Every algorithm is a loop over one chunk at a time (Section 3.3), so the
// chunk that starts at s depends only on bytes up to a horizon: RAM and AE
// read [s, s + max) and cut at s + max at the latest; MAXP also tests the w
// bytes right of a target (Section 2.1), so it reads [s - w, s + max + w).
// Once the bytes received reach s + H (H = max, plus w for MAXP) the chunk
// from s is the same whatever follows, and the feed emits it. The rest -- the
// bytes from the first start it cannot settle yet, with w bytes of left
// context for MAXP -- stays in a device staging buffer; the next piece is
// appended behind it and the staged bytes are chunked again from that start
// (cdc::chunk_in_context). The emitted lists of all pieces, concatenated,
// equal the boundaries of the whole stream chunked in one call.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cdc.h"
#include "cdc_launch.h"

struct cdc_feed_s {
    cdc_handle h = nullptr;
    cdc_alg alg = CDC_RAM;
    cdc_params p{};
    int device = 0;
    uint64_t horizon = 0;   // H
    uint64_t keep_ctx = 0;  // left context kept before the next start (MAXP: w)
    uint8_t* stg[2] = {nullptr, nullptr};  // staging, ping-pong
    size_t stg_cap[2] = {0, 0};
    int cur = 0;
    uint64_t ctx_lo = 0;    // stream offset of stg[cur][0]
    uint64_t carry = 0;     // stream offset where the next chunk starts
    uint64_t end = 0;       // bytes received
    bool done = false;      // the final piece was processed
    uint64_t* tmp = nullptr;  // boundaries of the staged bytes (relative to the carry)
    size_t tmp_cap = 0;       // elements
    uint64_t* d_info = nullptr;  // {boundaries settled, start of the first unsettled chunk, count}
    uint64_t* h_info = nullptr;  // page-locked copy
    cudaEvent_t staged = nullptr;  // the last copy into staging is done
};

namespace {

// Boundary i of b[0, total) closes the chunk that starts at b[i-1] (0 for
// i = 0). It is settled when that start + H <= rel (or on the final piece).
// Starts increase, so the settled ones are a prefix: one thread per block
// binary-searches its length, then the grid writes b + base to out.
__global__ void k_feed_settle(const uint64_t* b, uint64_t rel, uint64_t H, int final_piece, uint64_t base,
                              uint64_t* out, uint64_t cap, uint64_t* info) {
    __shared__ unsigned long long s_nf;
    if (threadIdx.x == 0) {
        const uint64_t total = info[2];  // written by the chain stage
        uint64_t nf = total;
        if (!final_piece) {
            uint64_t lo = 0, hi = total;
            while (lo < hi) {
                const uint64_t mid = lo + (hi - lo) / 2;
                const uint64_t start = mid ? b[mid - 1] : 0;
                if (start + H <= rel) lo = mid + 1;
                else hi = mid;
            }
            nf = lo;
        }
        s_nf = nf;
        if (blockIdx.x == 0) {
            info[0] = nf;
            info[1] = nf ? b[nf - 1] : 0;
        }
    }
    __syncthreads();
    const uint64_t nf = s_nf, lim = nf < cap ? nf : cap;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < lim; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = b[i] + base;
}

bool feed_params_ok(cdc_alg alg, cdc_params p) {
    if ((int)alg < 0 || (int)alg > 3) return false;
    if (p.w < 1 || p.min < 1 || p.min > p.max) return false;
    if (alg != CDC_MAXP && p.w >= p.max) return false;
    return true;
}

// grow a device buffer to `need` bytes, keeping its first `keep` bytes
cdc_status reserve(uint8_t** ptr, size_t* cap, size_t need, size_t keep, cudaStream_t st) {
    if (need <= *cap) return CDC_OK;
    size_t nc = need + need / 4 + (1u << 20);
    uint8_t* np = nullptr;
    if (cudaMalloc(&np, nc) != cudaSuccess) {
        cudaGetLastError();
        return CDC_ERR_NOMEM;
    }
    if (keep && cudaMemcpyAsync(np, *ptr, keep, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        cudaFree(np);
        return CDC_ERR_CUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaFree(np);
        return CDC_ERR_CUDA;
    }
    cudaFree(*ptr);
    *ptr = np;
    *cap = nc;
    return CDC_OK;
}

}  // namespace

extern "C" cdc_status cdc_feed_create(cdc_feed* out, cdc_handle h, cdc_alg alg, cdc_params p) {
    if (!out || !h || !feed_params_ok(alg, p)) return CDC_ERR_INVALID;
    *out = nullptr;
    cdc_feed f = new cdc_feed_s;
    f->h = h;
    f->alg = alg;
    f->p = p;
    cudaGetDevice(&f->device);
    f->horizon = (uint64_t)p.max + (alg == CDC_MAXP ? (uint64_t)p.w : 0);
    f->keep_ctx = alg == CDC_MAXP ? p.w : 0;
    if (cudaMalloc(&f->d_info, 3 * sizeof(uint64_t)) != cudaSuccess ||
        cudaMallocHost(&f->h_info, 3 * sizeof(uint64_t)) != cudaSuccess ||
        cudaEventCreateWithFlags(&f->staged, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cdc_feed_destroy(f);
        return CDC_ERR_NOMEM;
    }
    *out = f;
    return CDC_OK;
}

extern "C" cdc_status cdc_feed_destroy(cdc_feed f) {
    if (!f) return CDC_OK;
    cudaSetDevice(f->device);
    cudaDeviceSynchronize();
    cudaFree(f->stg[0]);
    cudaFree(f->stg[1]);
    cudaFree(f->tmp);
    cudaFree(f->d_info);
    cudaFreeHost(f->h_info);
    if (f->staged) cudaEventDestroy(f->staged);
    delete f;
    return CDC_OK;
}

extern "C" cdc_status cdc_feed_reset(cdc_feed f) {
    if (!f) return CDC_ERR_INVALID;
    cudaSetDevice(f->device);
    if (cudaEventSynchronize(f->staged) != cudaSuccess) return CDC_ERR_CUDA;
    f->cur = 0;
    f->ctx_lo = f->carry = f->end = 0;
    f->done = false;
    return CDC_OK;
}

extern "C" cdc_status cdc_feed_position(cdc_feed f, uint64_t* received, uint64_t* next_start) {
    if (!f) return CDC_ERR_INVALID;
    if (received) *received = f->end;
    if (next_start) *next_start = f->carry;
    return CDC_OK;
}

extern "C" cdc_status cdc_feed_push(cdc_feed f, const uint8_t* piece, size_t len, int final_piece,
                                    uint64_t* out_bounds, size_t* n, cdc_stream stream) {
    if (!f || !n || (len && !piece) || (*n && !out_bounds)) return CDC_ERR_INVALID;
    if (f->done) return CDC_ERR_INVALID;  // nothing may follow the final piece
    cudaSetDevice(f->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cap = *n;
    *n = 0;
    cdc_status s;
    // the previous push's last copy into staging may have run on another stream
    if (cudaStreamWaitEvent(st, f->staged, 0) != cudaSuccess) return CDC_ERR_CUDA;
    const uint64_t used = f->end - f->ctx_lo;
    if (len) {
        if ((s = reserve(&f->stg[f->cur], &f->stg_cap[f->cur], used + len, used, st)) != CDC_OK) return s;
        if (cudaMemcpyAsync(f->stg[f->cur] + used, piece, len, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return CDC_ERR_CUDA;
        f->end += len;
    }
    if (!final_piece && f->carry + f->horizon > f->end) {  // nothing settles yet
        if (cudaEventRecord(f->staged, st) != cudaSuccess) return CDC_ERR_CUDA;
        return cudaStreamSynchronize(st) == cudaSuccess ? CDC_OK : CDC_ERR_CUDA;
    }
    const uint64_t rel = f->end - f->carry, ctx = f->carry - f->ctx_lo;
    if (rel == 0) {  // final piece, nothing left after the last boundary
        f->done = true;
        return CDC_OK;
    }
    const size_t bound = rel / f->p.min + 2;  // chunks other than the last are >= min
    if (bound > f->tmp_cap) {
        uint8_t* t = reinterpret_cast<uint8_t*>(f->tmp);
        size_t tc = f->tmp_cap * sizeof(uint64_t);
        if ((s = reserve(&t, &tc, bound * sizeof(uint64_t), 0, st)) != CDC_OK) return s;
        f->tmp = reinterpret_cast<uint64_t*>(t);
        f->tmp_cap = tc / sizeof(uint64_t);
    }
    s = cdc::chunk_in_context(f->h, f->alg, f->p, f->stg[f->cur] + ctx, rel, ctx, f->tmp, f->tmp_cap,
                              f->d_info + 2, st);
    if (s != CDC_OK) return s;
    uint64_t grid = (bound + 255) / 256;
    if (grid > 1024) grid = 1024;
    k_feed_settle<<<(unsigned)grid, 256, 0, st>>>(f->tmp, rel, f->horizon, final_piece ? 1 : 0, f->carry,
                                                  out_bounds, cap, f->d_info);
    if (cudaGetLastError() != cudaSuccess) return CDC_ERR_CUDA;
    if (cudaMemcpyAsync(f->h_info, f->d_info, 3 * sizeof(uint64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return CDC_ERR_CUDA;
    if ((s = cdc::handle_status(f->h, st)) != CDC_OK) return s;  // the one synchronisation of a push
    const uint64_t nf = f->h_info[0], next_rel = f->h_info[1];
    if (f->h_info[2] > f->tmp_cap) return CDC_ERR_INTERNAL;  // more chunks than rel / min + 2: cannot happen
    *n = (size_t)nf;
    if (nf > cap) return CDC_ERR_CAPACITY;  // the piece stays staged: push again (len 0) with more room
    if (final_piece) {
        f->carry = f->end;
        f->done = true;
        return CDC_OK;
    }
    // keep [next start - context, end) at the start of the other staging buffer
    const uint64_t nc = f->carry + next_rel;
    const uint64_t nlo = nc - (nc < f->keep_ctx ? nc : f->keep_ctx);
    const uint64_t keep = f->end - nlo;
    const int o = f->cur ^ 1;
    if ((s = reserve(&f->stg[o], &f->stg_cap[o], keep, 0, st)) != CDC_OK) return s;
    if (cudaMemcpyAsync(f->stg[o], f->stg[f->cur] + (nlo - f->ctx_lo), keep, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess ||
        cudaEventRecord(f->staged, st) != cudaSuccess)
        return CDC_ERR_CUDA;
    f->cur = o;
    f->ctx_lo = nlo;
    f->carry = nc;
    return CDC_OK;
}
