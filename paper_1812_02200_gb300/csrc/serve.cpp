// serve.cpp -- the serving loop: many readouts, buffers arriving at random
// times, continuous batching under a device-memory budget.
//
// The paper's host runtime hands acquired buffers from the Rx thread to a
// processing thread through lock-free queues of pointers into pre-allocated
// memory (Sec. III).  Here:
//   - rfr_server_submit (any client thread) appends a request to a submission
//     queue and returns at once;
//   - one worker thread admits requests in arrival order as device memory
//     frees up: each request takes its input staging (host input) and output
//     staging from a pre-allocated arena the size of the budget (first-fit,
//     coalescing free list; no cudaMalloc while serving);
//   - an admitted request is enqueued immediately on its readout's stream
//     (H2D copy, the plan's push, copy of the frames to the client's buffers,
//     completion event), so work that arrives while other requests are on the
//     GPU overlaps with them (continuous batching); a readout's requests stay
//     in order because they share one stream, which also keeps its filter
//     history and NCO phase consistent on the device;
//   - completions (event done) release their memory and are reported through
//     rfr_server_poll with submit/admit/done timestamps; each request also
//     copies its plan's device status word to pinned host memory (and clears
//     it) before its event, so a device-side wait that gave up during that
//     request is reported as that request's RFR_E_TIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "dev_common.cuh"
#include "rfr_internal.h"
#include "trace.h"

namespace {

double now_us() {
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

// First-fit arena over one device allocation; offsets aligned to 256 B.
class Arena {
public:
    bool init(size_t bytes) {
        if (cudaMalloc(&base_, bytes) != cudaSuccess) {
            base_ = nullptr;
            return false;
        }
        size_ = bytes;
        free_[0] = bytes;
        return true;
    }
    ~Arena() {
        if (base_) cudaFree(base_);
    }
    // returns offset or SIZE_MAX
    size_t alloc(size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        if (bytes == 0) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, rem = it->second - bytes;
                free_.erase(it);
                if (rem) free_[off + bytes] = rem;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        if (bytes == 0) bytes = 256;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char* ptr(size_t off) const { return static_cast<char*>(base_) + off; }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

private:
    void* base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

struct Request {
    int32_t readout;
    const int16_t* iq;
    int64_t n;
    rfr_output out;
    uint64_t tag;
    double t_submit;
};

struct InFlight {
    Request rq;
    size_t off = 0, bytes = 0;
    int slot = -1;          // index of its completion event and status snapshot
    int64_t frames = 0;
    double t_admit = 0;
};

}  // namespace

struct rfr_server {
    std::vector<rfr_plan*> plans;
    std::vector<cudaStream_t> streams;
    Arena arena;
    int64_t max_samples = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> submitted;          // guarded by mu
    std::deque<rfr_completion> done;        // guarded by mu
    std::deque<Request> waiting;            // worker only
    std::vector<InFlight> in_flight;        // worker only
    std::vector<cudaEvent_t> events;        // one per slot
    int* h_status = nullptr;                // pinned: device status word per slot
    std::vector<int> free_slots;            // worker only
    std::atomic<bool> stop{false};
    std::thread worker;
    std::atomic<int64_t> n_submitted{0}, n_admitted{0}, n_completed{0}, n_queued{0}, n_inflight{0};
    std::string last_error;
    rfr_status error = RFR_OK;
};

namespace {

// Rows of row_bytes (a multiple of 8) from device memory src (pitch
// src_pitch) to dst (pitch dst_pitch), 8 bytes per thread and step: dst may
// be the device address of mapped pinned host memory, which the kernel
// writes directly.  The tone rows of one request are as short as its frame
// count (1-32 KB for the workload's buffers), and a 2-D copy-engine transfer
// of rows that short runs far below the host link's rate.
__global__ void copy_rows_kernel(char* __restrict__ dst, int64_t dst_pitch, const char* __restrict__ src,
                                 int64_t src_pitch, int64_t row_bytes, int64_t rows) {
    const int64_t words = row_bytes / 8;
    const int64_t total = words * rows;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = i / words, c = i - r * words;
        reinterpret_cast<uint64_t*>(dst + r * dst_pitch)[c] = reinterpret_cast<const uint64_t*>(src + r * src_pitch)[c];
    }
}

// Device address of pinned host memory, or nullptr (pageable, or device memory).
void* mapped_host(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return a.devicePointer;
}

bool host_pointer(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// Bytes of device staging one request needs: input (host input only) + the
// frames it will produce, laid out like the caller's buffers.
size_t request_bytes(const rfr_plan* p, const Request& r, int64_t F, bool host_in) {
    size_t b = host_in ? static_cast<size_t>(r.n) * 4 + 256 : 0;
    const int nt = static_cast<int>(p->words.size());
    if (p->mode == RFR_MODE_PFB && (p->out_flags & RFR_OUT_FULL)) b += static_cast<size_t>(F) * p->N * 8 + 256;
    if (nt > 0 && (p->mode == RFR_MODE_DEMOD || (p->out_flags & RFR_OUT_TONES)))
        b += static_cast<size_t>(F) * nt * 8 + 256;
    return b;
}

void worker_loop(rfr_server* s) {
    cudaSetDevice(s->device);
    while (true) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->submitted.empty() && s->waiting.empty() && s->in_flight.empty()) {
                if (s->stop.load()) break;
                s->cv.wait_for(lk, std::chrono::microseconds(200));
            }
            while (!s->submitted.empty()) {
                s->waiting.push_back(s->submitted.front());
                s->submitted.pop_front();
            }
        }
        // admission in arrival order while memory allows
        while (!s->waiting.empty() && !s->free_slots.empty()) {
            Request& rq = s->waiting.front();
            rfr_plan* p = s->plans[rq.readout];
            const bool host_in = rq.n > 0 && host_pointer(rq.iq);
            const int64_t F = rfr::frames_for_samples(p, rq.n);
            const size_t need = request_bytes(p, rq, F, host_in);
            const size_t off = s->arena.alloc(need);
            if (off == SIZE_MAX) break;   // head of the queue waits for memory
            InFlight f;
            f.rq = rq;
            f.off = off;
            f.bytes = need;
            f.frames = F;
            f.t_admit = now_us();
            rfr::TraceRange tr("rfr_server_admit");
            f.slot = s->free_slots.back();
            s->free_slots.pop_back();
            cudaStream_t st = s->streams[rq.readout];
            char* cur = s->arena.ptr(off);
            const int16_t* dev_in = rq.iq;
            if (host_in) {
                cudaMemcpyAsync(cur, rq.iq, static_cast<size_t>(rq.n) * 4, cudaMemcpyHostToDevice, st);
                dev_in = reinterpret_cast<const int16_t*>(cur);
                cur += (static_cast<size_t>(rq.n) * 4 + 255) & ~size_t(255);
            }
            rfr_output so{};
            const int nt = static_cast<int>(p->words.size());
            const bool want_full = p->mode == RFR_MODE_PFB && (p->out_flags & RFR_OUT_FULL);
            const bool want_tones = nt > 0 && (p->mode == RFR_MODE_DEMOD || (p->out_flags & RFR_OUT_TONES));
            if (want_full) {
                so.full = cur;
                so.full_ld = p->N;
                so.full_cap = F;
                cur += (static_cast<size_t>(F) * p->N * 8 + 255) & ~size_t(255);
            }
            if (want_tones) {
                so.tones = cur;
                so.tones_ld = std::max<int64_t>(F, 1);
                so.tones_cap = F;
            }
            int64_t got = 0;
            rfr_status rs = rfr::push_core(p, dev_in, rq.n, &so, &got, st);
            if (rs == RFR_OK && got > 0) {
                const rfr_output& o = rq.out;
                if (want_full)
                    cudaMemcpy2DAsync(static_cast<char*>(o.full) + o.frame_offset * o.full_ld * 8, o.full_ld * 8,
                                      so.full, static_cast<size_t>(p->N) * 8, static_cast<size_t>(p->N) * 8, got,
                                      cudaMemcpyDefault, st);
                if (want_tones) {
                    char* dst = static_cast<char*>(o.tones) + o.frame_offset * 8;
                    char* dmap = static_cast<char*>(mapped_host(o.tones));
                    if (dmap) {
                        // pinned host rows written by a kernel through the mapping
                        const int64_t total = got * nt;
                        const unsigned grid = static_cast<unsigned>(
                            std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, static_cast<int64_t>(p->n_sms) * 8)));
                        copy_rows_kernel<<<grid, 256, 0, st>>>(dmap + o.frame_offset * 8, o.tones_ld * 8,
                                                               static_cast<const char*>(so.tones), so.tones_ld * 8,
                                                               got * 8, nt);
                    } else {
                        cudaMemcpy2DAsync(dst, o.tones_ld * 8, so.tones, so.tones_ld * 8, got * 8, nt,
                                          cudaMemcpyDefault, st);
                    }
                }
            }
            if (rs != RFR_OK) {
                s->error = rs;
                s->last_error = p->last_error;
            }
            // this request's device status (a bounded wait that gave up),
            // then cleared so the readout's next request starts clean
            cudaMemcpyAsync(&s->h_status[f.slot], p->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
            cudaMemsetAsync(p->d_status, 0, sizeof(int), st);
            cudaEventRecord(s->events[f.slot], st);
            f.frames = rs == RFR_OK ? got : 0;
            s->in_flight.push_back(f);
            s->waiting.pop_front();
            s->n_admitted++;
        }
        s->n_queued = static_cast<int64_t>(s->waiting.size());
        // completions
        for (size_t i = 0; i < s->in_flight.size();) {
            InFlight& f = s->in_flight[i];
            const cudaError_t q = cudaEventQuery(s->events[f.slot]);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            rfr_completion c{};
            c.tag = f.rq.tag;
            c.readout = f.rq.readout;
            c.status = q == cudaSuccess ? RFR_OK : RFR_E_CUDA;
            if (q != cudaSuccess) cudaGetLastError();
            const int dev_status = s->h_status[f.slot];
            if (c.status == RFR_OK && dev_status == rfr::DEV_TIMEOUT) c.status = RFR_E_TIMEOUT;
            else if (c.status == RFR_OK && dev_status != rfr::DEV_OK) c.status = RFR_E_CUDA;
            c.frames = f.frames;
            c.samples = f.rq.n;
            c.t_submit_us = f.rq.t_submit;
            c.t_admit_us = f.t_admit;
            c.t_done_us = now_us();
            s->arena.release(f.off, f.bytes);
            s->free_slots.push_back(f.slot);
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->done.push_back(c);
            }
            s->n_completed++;
            s->in_flight[i] = s->in_flight.back();
            s->in_flight.pop_back();
        }
        s->n_inflight = static_cast<int64_t>(s->in_flight.size());
        if (!s->in_flight.empty() && s->waiting.empty()) std::this_thread::yield();
    }
}

void server_free(rfr_server* s) {
    if (!s) return;
    for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
    for (auto e : s->events)
        if (e) cudaEventDestroy(e);
    if (s->h_status) cudaFreeHost(s->h_status);
    delete s;
}

}  // namespace

extern "C" {

double rfr_now_us(void) { return now_us(); }

rfr_status rfr_server_create(rfr_server** out, rfr_plan* const* plans, int32_t n, size_t mem_budget_bytes,
                             int64_t max_buffer_samples) {
    if (!out || !plans || n < 1 || n > 4096 || mem_budget_bytes < (1u << 20) || max_buffer_samples < 1)
        return RFR_E_INVALID;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return RFR_E_INVALID;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return RFR_E_INVALID;
    }
    rfr_server* s = new (std::nothrow) rfr_server();
    if (!s) return RFR_E_NOMEM;
    cudaGetDevice(&s->device);
    s->plans.assign(plans, plans + n);
    s->max_samples = max_buffer_samples;
    // pre-size every plan's scratch so serving never allocates
    for (auto* p : s->plans) {
        if (rfr::ensure_scratch(p, max_buffer_samples) != RFR_OK) {
            server_free(s);
            return RFR_E_NOMEM;
        }
    }
    if (!s->arena.init(mem_budget_bytes)) {
        server_free(s);
        return RFR_E_NOMEM;
    }
    s->streams.resize(n, nullptr);
    for (auto& st : s->streams)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            server_free(s);
            return RFR_E_CUDA;
        }
    const size_t slots = static_cast<size_t>(n) * 8 + 64;
    s->events.resize(slots, nullptr);
    for (auto& e : s->events)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            server_free(s);
            return RFR_E_CUDA;
        }
    if (cudaHostAlloc(reinterpret_cast<void**>(&s->h_status), slots * sizeof(int), cudaHostAllocDefault) !=
        cudaSuccess) {
        s->h_status = nullptr;
        server_free(s);
        return RFR_E_NOMEM;
    }
    std::memset(s->h_status, 0, slots * sizeof(int));
    for (size_t i = 0; i < slots; ++i) s->free_slots.push_back(static_cast<int>(slots - 1 - i));
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return RFR_OK;
}

rfr_status rfr_server_submit(rfr_server* s, int32_t readout, const int16_t* iq, int64_t n,
                             const rfr_output* out, uint64_t tag) {
    if (!s || !out || readout < 0 || readout >= static_cast<int32_t>(s->plans.size())) return RFR_E_INVALID;
    if (n < 0 || n > s->max_samples || (n > 0 && !iq)) return RFR_E_INVALID;
    Request r{readout, iq, n, *out, tag, now_us()};
    // a request that could never fit in the budget would block the queue forever
    const rfr_plan* p = s->plans[readout];
    const int64_t f_max = (n + p->W) / p->H + 1;
    if (request_bytes(p, r, f_max, n > 0 && host_pointer(iq)) > s->arena.size()) return RFR_E_NOMEM;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->submitted.push_back(r);
    }
    s->n_submitted++;
    s->cv.notify_one();
    return RFR_OK;
}

rfr_status rfr_server_poll(rfr_server* s, rfr_completion* done, int32_t cap, int32_t* n_done, int32_t wait_ms) {
    if (!s || !n_done || (cap > 0 && !done)) return RFR_E_INVALID;
    *n_done = 0;
    const double deadline = now_us() + 1000.0 * std::max(wait_ms, 0);
    while (true) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            while (*n_done < cap && !s->done.empty()) {
                done[(*n_done)++] = s->done.front();
                s->done.pop_front();
            }
        }
        if (*n_done > 0 || now_us() >= deadline) break;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return s->error;
}

rfr_status rfr_server_get_stats(const rfr_server* s, rfr_server_stats* st) {
    if (!s || !st) return RFR_E_INVALID;
    st->submitted = s->n_submitted.load();
    st->admitted = s->n_admitted.load();
    st->completed = s->n_completed.load();
    st->queued = s->n_queued.load();
    st->in_flight = s->n_inflight.load();
    st->budget_bytes = static_cast<int64_t>(s->arena.size());
    st->peak_bytes = static_cast<int64_t>(s->arena.peak());
    return RFR_OK;
}

void rfr_server_destroy(rfr_server* s) {
    if (!s) return;
    s->stop = true;
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaDeviceSynchronize();
    server_free(s);
}

}  // extern "C"
