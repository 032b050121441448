// serve.cu -- the serving engine (include/cdc.h, cdc_server_*): chunking
// requests from host memory, admitted under a device-memory budget and run
// with continuous batching.
//
// A worker thread owns `slots` execution slots; each has a CUDA stream, a
// library handle (its workspace stays on the device between batches), a device
// arena for request bytes and a pinned staging area for offsets, copy
// descriptors and boundaries. Requests become eligible at their arrival time.
// Whenever a slot is free, the worker packs the eligible requests that share
// the oldest one's algorithm and parameters (oldest first, up to the slot's
// capacity) into one batch: requests in page-locked host memory (which the
// device reads directly) are listed as pieces of at most 64 KiB and brought in
// by one gather kernel; others take one host-to-device copy each; then one
// batched chunking call over the packed files, one copy of the boundary index
// and boundaries back, one event. Requests that arrive while slots are busy wait
// and join the next batch of their kind; batches on different slots overlap on
// the device (copies and kernels on separate streams). When a slot's event
// completes, the worker hands each request its boundaries and timestamps.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/cdc.h"
#include "cdc_launch.h"

namespace {

using Clock = std::chrono::steady_clock;

// One piece of a request to bring into the arena: `len` bytes (<= kPiece)
// from the device-addressable host address `src` to arena offset `dst`.
struct GatherPiece {
    const uint8_t* src;
    uint64_t dst;
    uint64_t len;
};
constexpr uint64_t kPiece = 64u << 10;
constexpr int kGatherThreads = 256;

// One CTA per piece: the destination's 16-byte granules inside the piece are
// stored whole (two aligned 16-byte loads of the source, funnel-shifted into
// place), the partial granules at its two ends byte by byte.
__global__ void __launch_bounds__(kGatherThreads) k_gather(const GatherPiece* pieces, uint32_t n, uint8_t* arena) {
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        const GatherPiece pc = pieces[i];
        const uint64_t d0 = pc.dst, d1 = pc.dst + pc.len;
        const uint64_t a0 = (d0 + 15) & ~15ull, a1 = d1 & ~15ull;  // whole granules [a0, a1)
        if (a0 >= a1) {
            for (uint64_t d = d0 + threadIdx.x; d < d1; d += kGatherThreads) arena[d] = pc.src[d - d0];
            continue;
        }
        for (uint64_t d = d0 + threadIdx.x; d < a0; d += kGatherThreads) arena[d] = pc.src[d - d0];
        for (uint64_t d = a1 + threadIdx.x; d < d1; d += kGatherThreads) arena[d] = pc.src[d - d0];
        for (uint64_t g = a0 + 16ull * threadIdx.x; g < a1; g += 16ull * kGatherThreads) {
            const uintptr_t sp = reinterpret_cast<uintptr_t>(pc.src) + (g - d0);
            const uint32_t sh = (uint32_t)(sp & 15);
            const uint4* q = reinterpret_cast<const uint4*>(sp - sh);
            const uint4 x = q[0];
            uint4 o;
            if (sh == 0) {
                o = x;
            } else {
                // the second granule holds the rest of this one's bytes, so it
                // lies in the source's pages
                const uint4 y = q[1];
                const uint32_t wv[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
                const uint32_t k = sh >> 2, r = 8 * (sh & 3);
                uint32_t ov[4];
#pragma unroll
                for (int j = 0; j < 4; j++) ov[j] = __funnelshift_r(wv[k + j], wv[k + j + 1], r);
                o = make_uint4(ov[0], ov[1], ov[2], ov[3]);
            }
            *reinterpret_cast<uint4*>(arena + g) = o;
        }
    }
}

struct Request {
    cdc_alg alg;
    cdc_params p;
    const uint8_t* data;
    const uint8_t* dev_src;  // the same bytes as the device addresses them (page-locked), or null
    size_t len;
    uint64_t* bounds;
    size_t capacity;
    uint64_t tag;
    double t_arrive, t_submit, t_start;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cdc_handle h = nullptr;
    cudaEvent_t done = nullptr;
    uint8_t* arena = nullptr;      // request bytes, packed
    uint64_t* d_off = nullptr;     // file offsets (max_files + 1)
    uint64_t* d_bounds = nullptr;  // boundaries
    uint64_t* d_index = nullptr;   // per-file boundary index (max_files + 1)
    uint64_t* h_off = nullptr;     // pinned staging
    GatherPiece* h_pieces = nullptr;  // pinned: copy descriptors of the batch
    GatherPiece* d_pieces = nullptr;
    size_t pieces_cap = 0;
    uint64_t* h_index = nullptr;
    uint64_t* h_bounds = nullptr;
    size_t bounds_cap = 0;
    std::vector<Request> batch;
    bool busy = false;
};

bool same_kind(const Request& a, const Request& b) {
    return a.alg == b.alg && a.p.w == b.p.w && a.p.min == b.p.min && a.p.max == b.p.max;
}

}  // namespace

struct cdc_server_s {
    int device = 0;
    size_t slot_bytes = 0;  // arena bytes per slot
    size_t max_files = 0;   // requests per batch
    std::vector<Slot> slots;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> inbox;        // submitted, not yet taken by the worker
    std::deque<cdc_result> done;      // finished, not yet polled
    std::condition_variable done_cv;
    std::atomic<bool> stop{false};
    std::atomic<int64_t> outstanding{0};
    std::thread worker;
    cdc_status fatal = CDC_OK;

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
    void run();
    bool launch(Slot& s, std::deque<Request>& pending, double now);
    void finish(Slot& s);
};

static void slot_free(Slot& s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.h) cdc_destroy(s.h);
    if (s.done) cudaEventDestroy(s.done);
    cudaFree(s.arena);
    cudaFree(s.d_off);
    cudaFree(s.d_bounds);
    cudaFree(s.d_index);
    if (s.h_off) cudaFreeHost(s.h_off);
    if (s.h_pieces) cudaFreeHost(s.h_pieces);
    cudaFree(s.d_pieces);
    if (s.h_index) cudaFreeHost(s.h_index);
    if (s.h_bounds) cudaFreeHost(s.h_bounds);
    if (s.stream) cudaStreamDestroy(s.stream);
    s = Slot();
}

// Pack eligible requests of the oldest one's kind into a batch on slot s.
bool cdc_server_s::launch(Slot& s, std::deque<Request>& pending, double now) {
    auto first = std::find_if(pending.begin(), pending.end(), [&](const Request& r) { return r.t_arrive <= now; });
    if (first == pending.end()) return false;
    const Request key = *first;
    s.batch.clear();
    size_t bytes = 0, nb = 0;
    // one pass: the requests taken go to the batch, the others (in order) to
    // `rest`, which becomes the pending queue (erasing from the middle of the
    // queue instead would cost time quadratic in its length)
    std::deque<Request> rest;
    bool open = true;
    for (auto it = pending.begin(); it != pending.end(); ++it) {
        if (open && it >= first && it->t_arrive <= now && same_kind(*it, key)) {
            const size_t need_b = it->len / it->p.min + 1;
            if (bytes + it->len <= slot_bytes && nb + need_b <= s.bounds_cap) {
                bytes += it->len;
                nb += need_b;
                s.batch.push_back(*it);
                if (s.batch.size() >= max_files) open = false;
                continue;
            }
            if (!s.batch.empty()) open = false;  // the batch is full (submit rejects requests larger than a slot)
        }
        rest.push_back(*it);
    }
    pending.swap(rest);
    if (s.batch.empty()) return false;
    const size_t n = s.batch.size();
    s.h_off[0] = 0;
    size_t np = 0;  // gather pieces
    for (size_t i = 0; i < n; i++) {
        Request& r = s.batch[i];
        r.t_start = now;
        s.h_off[i + 1] = s.h_off[i] + r.len;
        if (!r.len) continue;
        if (r.dev_src && np + (r.len + kPiece - 1) / kPiece <= s.pieces_cap) {
            for (uint64_t o = 0; o < r.len; o += kPiece)
                s.h_pieces[np++] = GatherPiece{r.dev_src + o, s.h_off[i] + o, std::min<uint64_t>(kPiece, r.len - o)};
        } else if (cudaMemcpyAsync(s.arena + s.h_off[i], r.data, r.len, cudaMemcpyHostToDevice, s.stream) !=
                   cudaSuccess) {
            fatal = CDC_ERR_CUDA;
        }
    }
    if (np) {
        if (cudaMemcpyAsync(s.d_pieces, s.h_pieces, np * sizeof(GatherPiece), cudaMemcpyHostToDevice, s.stream) !=
            cudaSuccess)
            fatal = CDC_ERR_CUDA;
        const unsigned grid = (unsigned)std::min<size_t>(np, 65535);
        k_gather<<<grid, kGatherThreads, 0, s.stream>>>(s.d_pieces, (uint32_t)np, s.arena);
        if (cudaGetLastError() != cudaSuccess) fatal = CDC_ERR_CUDA;
    }
    if (cudaMemcpyAsync(s.d_off, s.h_off, (n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s.stream) != cudaSuccess)
        fatal = CDC_ERR_CUDA;
    cdc_status st = cdc_chunk_batch(s.h, key.alg, key.p, s.arena, bytes, s.d_off, n, s.d_bounds, s.d_index,
                                    s.bounds_cap, nullptr, s.stream);
    if (st != CDC_OK) fatal = st;
    cudaMemcpyAsync(s.h_index, s.d_index, (n + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, s.stream);
    cudaMemcpyAsync(s.h_bounds, s.d_bounds, nb * sizeof(uint64_t), cudaMemcpyDeviceToHost, s.stream);
    cudaEventRecord(s.done, s.stream);
    s.busy = true;
    return true;
}

void cdc_server_s::finish(Slot& s) {
    cdc_status st = cdc_sync_status(s.h, s.stream);
    const double t = now_ms();
    std::vector<cdc_result> res;
    res.reserve(s.batch.size());
    for (size_t i = 0; i < s.batch.size(); i++) {
        const Request& r = s.batch[i];
        cdc_result o;
        memset(&o, 0, sizeof o);
        o.tag = r.tag;
        o.alg = (int32_t)r.alg;
        o.t_arrive_ms = r.t_arrive;
        o.t_submit_ms = r.t_submit;
        o.t_start_ms = r.t_start;
        o.t_done_ms = t;
        o.batch_size = (uint32_t)s.batch.size();
        if (st != CDC_OK) {
            o.status = st;
        } else {
            const uint64_t k = s.h_index[i + 1] - s.h_index[i];
            o.n_bounds = k;
            if (k > r.capacity) {
                o.status = CDC_ERR_CAPACITY;
            } else {
                memcpy(r.bounds, s.h_bounds + s.h_index[i], k * sizeof(uint64_t));
                o.status = CDC_OK;
            }
        }
        res.push_back(o);
    }
    s.busy = false;
    s.batch.clear();
    {
        std::lock_guard<std::mutex> lock(mu);
        for (auto& o : res) done.push_back(o);
    }
    outstanding -= (int64_t)res.size();
    done_cv.notify_all();
}

void cdc_server_s::run() {
    cudaSetDevice(device);
    // `ready`: arrived requests in arrival order (what a batch is packed from);
    // `future`: requests whose arrival time lies ahead, sorted by it. Batching
    // scans only the arrived requests, however many are submitted ahead.
    std::deque<Request> ready, future;
    auto by_arrival = [](const Request& a, const Request& b) { return a.t_arrive < b.t_arrive; };
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(mu);
            const bool any_busy = std::any_of(slots.begin(), slots.end(), [](const Slot& s) { return s.busy; });
            if (inbox.empty() && !any_busy && ready.empty()) {
                if (future.empty()) {
                    if (stop) break;
                    cv.wait_for(lock, std::chrono::milliseconds(2));
                } else {
                    // waiting only for arrival times: sleep until the next one (or new work)
                    const double d = future.front().t_arrive - now_ms();
                    if (d > 0.05) cv.wait_for(lock, std::chrono::microseconds((int64_t)(d * 1000.0)));
                }
            }
            while (!inbox.empty()) {
                const Request& r = inbox.front();
                if (future.empty() || !by_arrival(r, future.back())) future.push_back(r);  // the usual case
                else future.insert(std::upper_bound(future.begin(), future.end(), r, by_arrival), r);
                inbox.pop_front();
            }
        }
        bool progress = false;
        for (Slot& s : slots) {
            if (s.busy && cudaEventQuery(s.done) == cudaSuccess) {
                finish(s);
                progress = true;
            }
        }
        const double t = now_ms();
        while (!future.empty() && future.front().t_arrive <= t) {
            ready.push_back(future.front());
            future.pop_front();
        }
        for (Slot& s : slots)
            if (!s.busy && !ready.empty() && launch(s, ready, t)) progress = true;
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    for (Slot& s : slots)
        if (s.busy) {
            cudaEventSynchronize(s.done);
            finish(s);
        }
}

// Device bytes a handle's workspace takes for a batch of `arena` bytes and
// up to nf files (the sizes cdc_reserve grows to, with grow()'s 25% slack).
static size_t workspace_bytes(size_t arena, size_t nf, int sms) {
    size_t seg = arena / ((size_t)(sms > 0 ? sms : 148) * 16 + nf);
    seg = std::min(std::max(seg, (size_t)32 << 10), (size_t)256 << 10);
    seg = (seg + 63) & ~(size_t)63;
    const size_t items = arena / seg + nf + 2;
    const size_t nblk = (arena + 127) / 64 + 16;
    size_t b = 2 * (nblk + 64) + arena / 4096 + 66;
    b += items * (cdc::seg_state_bytes() + cdc::seg_hash_bytes() + cdc::seg_log_bytes(cdc::HANDLE_LOG_CAP));
    b += ((items + 127) / 128 + 1) * cdc::group_state_bytes();
    b += (nf + 1) * 8 + cdc::batch_scan_tmp_elems(nf) * 8 + items * 4 + 4096;
    return b + b / 4 + 8 * 64 * 4;
}

extern "C" cdc_status cdc_server_create(cdc_server* out, int device, size_t budget_bytes, int slots,
                                        size_t max_batch) {
    if (!out || slots < 1 || slots > 64 || budget_bytes < ((size_t)64 << 20)) return CDC_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return CDC_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return CDC_ERR_CUDA;
    cdc_server s = new cdc_server_s();
    s->device = device;
    s->max_files = max_batch ? max_batch : 4096;
    // per slot: the arena, the boundary buffer and index, and the library's
    // workspace for a full arena must fit the slot's share of the budget
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const size_t share = budget_bytes / (size_t)slots;
    size_t arena = share / 4 * 3;
    for (int it = 0; it < 200; it++) {
        const size_t bc = arena / 1024 + s->max_files + 1;
        if (arena + workspace_bytes(arena, s->max_files, sms) + bc * 8 + 2 * (s->max_files + 1) * 8 <= share) break;
        arena = arena / 10 * 9;
    }
    s->slot_bytes = arena & ~(size_t)255;
    s->slots.resize((size_t)slots);
    const size_t bcap = s->slot_bytes / 1024 + s->max_files + 1;  // boundaries per batch
    const size_t pcap = s->slot_bytes / kPiece + s->max_files + 1;  // gather pieces per batch
    for (Slot& sl : s->slots) {
        sl.bounds_cap = bcap;
        sl.pieces_cap = pcap;
        bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
                  cdc_create(&sl.h, device) == CDC_OK && cudaMalloc(&sl.arena, s->slot_bytes) == cudaSuccess &&
                  cudaMalloc(&sl.d_off, (s->max_files + 1) * sizeof(uint64_t)) == cudaSuccess &&
                  cudaMalloc(&sl.d_index, (s->max_files + 1) * sizeof(uint64_t)) == cudaSuccess &&
                  cudaMalloc(&sl.d_bounds, bcap * sizeof(uint64_t)) == cudaSuccess &&
                  cudaMallocHost(&sl.h_off, (s->max_files + 1) * sizeof(uint64_t)) == cudaSuccess &&
                  cudaMallocHost(&sl.h_pieces, pcap * sizeof(GatherPiece)) == cudaSuccess &&
                  cudaMalloc(&sl.d_pieces, pcap * sizeof(GatherPiece)) == cudaSuccess &&
                  cudaMallocHost(&sl.h_index, (s->max_files + 1) * sizeof(uint64_t)) == cudaSuccess &&
                  cudaMallocHost(&sl.h_bounds, bcap * sizeof(uint64_t)) == cudaSuccess;
        // the workspace for a full slot, so batches do not allocate
        if (ok) ok = cdc_reserve(sl.h, CDC_RAM, cdc_params{64, 64, 65536}, s->slot_bytes, s->max_files) == CDC_OK;
        if (!ok) {
            cudaGetLastError();
            for (Slot& t : s->slots) slot_free(t);
            delete s;
            return CDC_ERR_NOMEM;
        }
    }
    s->t0 = Clock::now();
    s->worker = std::thread([s]() { s->run(); });
    *out = s;
    return CDC_OK;
}

extern "C" cdc_status cdc_server_submit(cdc_server s, cdc_alg alg, cdc_params p, const uint8_t* host_data, size_t len,
                                        uint64_t* host_bounds, size_t capacity, uint64_t tag, double arrive_ms) {
    if (!s || (!host_data && len) || (!host_bounds && capacity) || (int)alg < 0 || (int)alg > 3) return CDC_ERR_INVALID;
    if (p.w < 1 || p.min < 1 || p.min > p.max || (alg != CDC_MAXP && p.w >= p.max) || p.min < 64)
        return CDC_ERR_INVALID;
    if (len > s->slot_bytes || len / p.min + 1 > s->slots[0].bounds_cap) return CDC_ERR_CAPACITY;
    Request r;
    r.alg = alg;
    r.p = p;
    r.data = host_data;
    r.dev_src = nullptr;
    if (len) {
        // page-locked host memory: the device reads it directly (one gather
        // kernel per batch instead of a copy call per request)
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, host_data) == cudaSuccess && at.type == cudaMemoryTypeHost &&
            at.devicePointer)
            r.dev_src = static_cast<const uint8_t*>(at.devicePointer);
        else
            cudaGetLastError();
    }
    r.len = len;
    r.bounds = host_bounds;
    r.capacity = capacity;
    r.tag = tag;
    r.t_submit = s->now_ms();
    r.t_arrive = arrive_ms < r.t_submit ? r.t_submit : arrive_ms;
    r.t_start = 0;
    s->outstanding++;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->inbox.push_back(r);
    }
    s->cv.notify_one();
    return CDC_OK;
}

extern "C" cdc_status cdc_server_poll(cdc_server s, cdc_result* out, int max, int* n, int wait_ms) {
    if (!s || !n || max < 0 || (!out && max)) return CDC_ERR_INVALID;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->done_cv.wait_for(lock, std::chrono::milliseconds(wait_ms), [&]() { return !s->done.empty(); });
    int k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n = k;
    return s->fatal;
}

extern "C" cdc_status cdc_server_clock(cdc_server s, double* now_ms) {
    if (!s || !now_ms) return CDC_ERR_INVALID;
    *now_ms = s->now_ms();
    return CDC_OK;
}

extern "C" cdc_status cdc_server_destroy(cdc_server s) {
    if (!s) return CDC_OK;
    s->stop = true;
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (Slot& sl : s->slots) slot_free(sl);
    delete s;
    return CDC_OK;
}
