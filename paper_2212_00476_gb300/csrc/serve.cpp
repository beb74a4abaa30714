// serve.cpp -- the serving layer of libzncc (serve_* in include/zncc.h): a queue of stereo
// requests from host memory, admitted under a device-memory budget onto a pool of contexts
// and run by continuous batching: whenever requests wait and slots are free, the scheduler
// thread launches the waiting small ones that share DT parameters as one zncc_run_batch (up
// to 32 pairs of uneven sizes), and a pair large enough to fill the GPU by itself alone, so
// that a new launch starts while earlier ones are still on the GPU. Large pairs go to a
// high-priority stream, in arrival order, batches of small pairs to a low-priority one: the
// block scheduler then gives a large pair the SMs as they free up and the small batches fill
// the gaps, so that two large pairs never share the GPU (each would finish as late as the
// pair of them in sequence) and a large pair never waits behind small ones.
// Completion is signalled by a host function queued behind each batch's result copies.
//
// Contexts (and their image, disparity and volume buffers) are kept per request shape and
// reused; idle ones are evicted, least recently used first, when a new shape needs room.
// Every wait of the host side is bounded: serve_poll by its timeout, serve_destroy by
// kDrainSeconds.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "zncc.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kMaxQueued = 1 << 16;     // requests waiting or running at once
constexpr double kDrainSeconds = 30.0;     // serve_destroy's bound on in-flight work
// A pair of at least this many volume elements fills the GPU by itself: it runs alone, with
// the single-pair kernels; smaller ones are batched together.
constexpr long long kAloneElements = 1LL << 25;

bool runs_alone(int W, int H, int D) { return (long long)W * H * D >= kAloneElements; }

struct ShapeKey {
    int W, H, D, win, storage, iters;
    bool operator==(const ShapeKey& o) const {
        return W == o.W && H == o.H && D == o.D && win == o.win && storage == o.storage && iters == o.iters;
    }
};

// Device bytes a context of this shape holds: DT coefficients (two float4 per pixel), the
// fused WTA's keys, the volume (pixel stride padded to 4 entries), the A_hat maps and
// multipliers of the F16 and I8 paths, the images and map.
size_t shape_charge(const ShapeKey& k) {
    const size_t npix = (size_t)k.W * k.H;
    size_t b = 32 * npix + 8 * npix + 4 * npix;
    if (k.iters > 0) {
        b += npix * (size_t)((k.D + 3) / 4 * 4) * (k.storage == ZNCC_F32 ? 4 : (k.storage == ZNCC_F16 ? 2 : 1));
        if (k.storage == ZNCC_F16 && k.iters > 1) b += npix * 12 * (size_t)(2 * k.iters - 1);
        if (k.storage == ZNCC_I8) b += npix * (4 * (size_t)(2 * k.iters - 1) + 8 * (size_t)(2 * k.iters));
    }
    return b;
}

struct Slot {
    ShapeKey key;
    zncc_ctx* ctx = nullptr;
    uint8_t* d_img = nullptr;      // [2][H][W]: left, right
    uint16_t* d_disp = nullptr;    // [H][W]
    size_t charge = 0;
    bool busy = false;
    uint64_t last_use = 0;
};

struct HostBuf {
    void* p = nullptr;
    size_t bytes = 0;
    bool pinned = false;
};

// The CUDA events of one batch (uploads start, uploads done, run done, copies done), shared
// by its requests; the last request polled returns them to the server's pool.
struct BatchTiming {
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool recorded = false;
    int refs = 0, pairs = 0;
};

struct Request {
    uint64_t ticket = 0;
    ShapeKey key{};
    float sigma_s = 0.f, sigma_r = 0.f;
    HostBuf img, disp;             // [2][H][W] uint8 inputs, [H][W] uint16 result
    enum State { QUEUED, RUNNING, DONE } state = QUEUED;
    zncc_status status = ZNCC_OK;
    Slot* slot = nullptr;
    Clock::time_point t_submit, t_issue, t_done;
    BatchTiming* timing = nullptr;
};

}  // namespace

struct zncc_server {
    size_t budget = 0;
    int max_slots = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;            // state changes: submissions, completions, stop
    std::deque<Request*> queue;            // waiting, in submission order
    std::unordered_map<uint64_t, Request*> tickets;
    std::vector<Slot*> slots;
    std::multimap<size_t, HostBuf> free_bufs;   // host buffers for reuse, by size
    std::vector<cudaEvent_t> free_events;         // timing events for reuse
    size_t charged = 0;
    int inflight = 0;                      // requests on the GPU
    uint64_t next_ticket = 1, use_clock = 0, completions = 0;
    bool stopping = false, thread_done = false;
    cudaStream_t streams[2] = {nullptr, nullptr};   // large pairs (high priority), batches (low)
    char err[512] = {0};
    std::thread worker;
};

namespace {

struct Batch {
    zncc_server* s;
    std::vector<Request*> reqs;
};

void set_err(zncc_server* s, const char* fmt, const char* a = "", const char* b = "") {
    snprintf(s->err, sizeof(s->err), fmt, a, b);
}

// Host buffers: pinned when the runtime can provide them (asynchronous copies), else plain
// memory (the copies then run synchronously with the host). Reused by size: pool_take
// (under the lock) returns an empty buffer when none is free, new_buf allocates one.
HostBuf pool_take(zncc_server* s, size_t bytes) {
    auto it = s->free_bufs.find(bytes);
    if (it == s->free_bufs.end()) return HostBuf();
    HostBuf b = it->second;
    s->free_bufs.erase(it);
    return b;
}

HostBuf new_buf(size_t bytes) {
    HostBuf b;
    b.bytes = bytes;
    if (cudaHostAlloc(&b.p, bytes, cudaHostAllocPortable) == cudaSuccess) {
        b.pinned = true;
    } else {
        cudaGetLastError();
        b.p = malloc(bytes);
    }
    return b;
}

void drop_buf(const HostBuf& b) {
    if (!b.p) return;
    if (b.pinned) cudaFreeHost(b.p);
    else free(b.p);
}

void give_buf(zncc_server* s, HostBuf& b) {
    if (b.p) s->free_bufs.emplace(b.bytes, b);
    b = HostBuf();
}

void destroy_slot(Slot* sl) {
    if (sl->ctx) zncc_destroy(sl->ctx);
    if (sl->d_img) cudaFree(sl->d_img);
    if (sl->d_disp) cudaFree(sl->d_disp);
    delete sl;
}

// An idle slot of this shape, taken (busy), or nullptr. Under the lock.
Slot* take_idle(zncc_server* s, const ShapeKey& key) {
    for (Slot* sl : s->slots)
        if (!sl->busy && sl->key == key) {
            sl->busy = true;
            return sl;
        }
    return nullptr;
}

// Reserves `need` bytes of the budget, taking idle slots out of the pool, least recently
// used first, until they fit; the caller destroys `victims` after releasing the lock.
// False (nothing changed) when even every idle slot would not make room. Under the lock.
bool reserve(zncc_server* s, size_t need, std::vector<Slot*>& victims) {
    std::vector<Slot*> idle;
    for (Slot* sl : s->slots)
        if (!sl->busy) idle.push_back(sl);
    std::sort(idle.begin(), idle.end(), [](const Slot* a, const Slot* b) { return a->last_use < b->last_use; });
    size_t freed = 0;
    size_t k = 0;
    while (s->charged - freed + need > s->budget && k < idle.size()) freed += idle[k++]->charge;
    if (s->charged - freed + need > s->budget) return false;
    for (size_t i = 0; i < k; ++i) {
        victims.push_back(idle[i]);
        s->slots.erase(std::find(s->slots.begin(), s->slots.end(), idle[i]));
    }
    s->charged = s->charged - freed + need;
    return true;
}

// A new context and its buffers for this shape, or nullptr with *st set. Makes CUDA calls
// that may synchronize the device: never under the lock (a batch's completion function
// needs the lock, so waiting for the device while holding it would never end).
Slot* create_slot(const ShapeKey& key, size_t charge, zncc_status* st, char* err, size_t errlen) {
    Slot* sl = new Slot();
    sl->key = key;
    sl->charge = charge;
    const size_t npix = (size_t)key.W * key.H;
    *st = zncc_create(key.W, key.H, key.D, key.win, &sl->ctx);
    if (*st != ZNCC_OK) {
        snprintf(err, errlen, "context for a request: %s", zncc_last_error(nullptr));
    } else {
        cudaError_t e = zncc::device_alloc((void**)&sl->d_img, 2 * npix);
        if (e == cudaSuccess) e = zncc::device_alloc((void**)&sl->d_disp, npix * sizeof(uint16_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            *st = e == cudaErrorMemoryAllocation ? ZNCC_ENOMEM : ZNCC_ECUDA;
            snprintf(err, errlen, "image buffers of a request: %s", cudaGetErrorString(e));
        }
    }
    if (*st != ZNCC_OK) {
        destroy_slot(sl);
        return nullptr;
    }
    sl->busy = true;
    return sl;
}

void finish(zncc_server* s, Request* r, zncc_status st) {
    r->status = st;
    r->state = Request::DONE;
    r->t_done = Clock::now();
    if (r->slot) {
        r->slot->busy = false;
        r->slot->last_use = ++s->use_clock;
        r->slot = nullptr;
    }
}

// Runs behind a batch's result copies on its stream (a CUDA host function: no CUDA calls).
void CUDART_CB on_batch_done(void* p) {
    Batch* b = static_cast<Batch*>(p);
    zncc_server* s = b->s;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Request* r : b->reqs) finish(s, r, ZNCC_OK);
        s->inflight -= (int)b->reqs.size();
        ++s->completions;
    }
    s->cv.notify_all();
    delete b;
}

// Queues one batch: image uploads, the batched fused run, result downloads, completion.
// Called without the lock; on failure the batch's requests end with the error.
void launch(zncc_server* s, Batch* b) {
    const int n = (int)b->reqs.size();
    const Request* head = b->reqs[0];
    cudaStream_t st = s->streams[runs_alone(head->key.W, head->key.H, head->key.D) ? 0 : 1];
    zncc_ctx* ctxs[zncc::kMaxBatch];
    const uint8_t* lefts[zncc::kMaxBatch];
    const uint8_t* rights[zncc::kMaxBatch];
    int pitches[zncc::kMaxBatch];
    uint16_t* disps[zncc::kMaxBatch];
    zncc_status status = ZNCC_OK;
    cudaError_t e = cudaSuccess;
    // the batch's timing events, from the pool or created (outside the lock)
    BatchTiming* bt = new BatchTiming();
    bt->refs = n;
    bt->pairs = n;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int k = 0; k < 4 && !s->free_events.empty(); ++k) {
            bt->ev[k] = s->free_events.back();
            s->free_events.pop_back();
        }
    }
    bool timed = true;
    for (int k = 0; k < 4; ++k)
        if (!bt->ev[k] && cudaEventCreate(&bt->ev[k]) != cudaSuccess) {
            cudaGetLastError();
            bt->ev[k] = nullptr;
            timed = false;
        }
    const Clock::time_point t_issue = Clock::now();
    for (Request* r : b->reqs) {
        r->t_issue = t_issue;
        r->timing = bt;
    }
    if (timed) timed = cudaEventRecord(bt->ev[0], st) == cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        Request* r = b->reqs[i];
        Slot* sl = r->slot;
        const size_t npix = (size_t)r->key.W * r->key.H;
        e = cudaMemcpyAsync(sl->d_img, r->img.p, 2 * npix, cudaMemcpyHostToDevice, st);
        zncc_set_stream(sl->ctx, st);
        ctxs[i] = sl->ctx;
        lefts[i] = sl->d_img;
        rights[i] = sl->d_img + npix;
        pitches[i] = r->key.W;
        disps[i] = sl->d_disp;
    }
    if (timed && e == cudaSuccess) timed = cudaEventRecord(bt->ev[1], st) == cudaSuccess;
    if (e == cudaSuccess) {
        const Request* r0 = b->reqs[0];
        status = zncc_run_batch(ctxs, lefts, rights, pitches, disps, n, r0->sigma_s, r0->sigma_r,
                                r0->key.iters, (zncc_dtype)r0->key.storage);
        if (status != ZNCC_OK) {
            std::lock_guard<std::mutex> lk(s->mu);
            set_err(s, "batched run: %s", zncc_last_error(ctxs[0]));
        }
    }
    if (timed && e == cudaSuccess && status == ZNCC_OK) timed = cudaEventRecord(bt->ev[2], st) == cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess && status == ZNCC_OK; ++i) {
        Request* r = b->reqs[i];
        e = cudaMemcpyAsync(r->disp.p, r->slot->d_disp, (size_t)r->key.W * r->key.H * sizeof(uint16_t),
                            cudaMemcpyDeviceToHost, st);
    }
    if (timed && e == cudaSuccess && status == ZNCC_OK) timed = cudaEventRecord(bt->ev[3], st) == cudaSuccess;
    if (!timed) cudaGetLastError();
    bt->recorded = timed;
    if (e == cudaSuccess && status == ZNCC_OK) e = cudaLaunchHostFunc(st, on_batch_done, b);
    if (e == cudaSuccess && status == ZNCC_OK) return;
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(s->mu);
        set_err(s, "batch launch: %s (%s)", cudaGetErrorName(e), cudaGetErrorString(e));
        status = ZNCC_ECUDA;
        cudaGetLastError();
    }
    cudaStreamSynchronize(st);        // nothing of the batch may still use its buffers
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Request* r : b->reqs) finish(s, r, status);
        s->inflight -= n;
        ++s->completions;
    }
    s->cv.notify_all();
    delete b;
}

// The scheduler thread: admit waiting requests in submission order while slots and budget
// allow, batch those that share the DT parameters and storage, launch, repeat.
void worker_main(zncc_server* s) {
    bool ok = cudaSetDevice(s->device) == cudaSuccess;
    int least = 0, greatest = 0;                  // numerically: greatest priority <= least
    if (ok) ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess;
    for (int i = 0; ok && i < 2; ++i)
        ok = cudaStreamCreateWithPriority(&s->streams[i], cudaStreamNonBlocking, i == 0 ? greatest : least) ==
             cudaSuccess;
    std::unique_lock<std::mutex> lk(s->mu);
    if (!ok) {
        cudaGetLastError();
        set_err(s, "scheduler set-up: no usable CUDA device");
    }
    uint64_t seen = s->completions;
    for (;;) {
        s->cv.wait(lk, [&] {
            return s->stopping || (!s->queue.empty() && s->inflight < s->max_slots &&
                                   (s->inflight == 0 || s->completions != seen || !ok));
        });
        if (s->stopping) break;
        seen = s->completions;
        if (!ok) {                                   // no device: every request fails
            while (!s->queue.empty()) {
                finish(s, s->queue.front(), ZNCC_ECUDA);
                s->queue.pop_front();
            }
            s->cv.notify_all();
            continue;
        }
        Batch* b = new Batch{s, {}};
        const Request* head = nullptr;
        size_t idx = 0;
        while (idx < s->queue.size() && (int)b->reqs.size() < zncc::kMaxBatch &&
               s->inflight + (int)b->reqs.size() < s->max_slots) {
            Request* r = s->queue[idx];
            const bool alone = runs_alone(r->key.W, r->key.H, r->key.D);
            if (head && alone) break;                           // a large pair starts its own launch
            if (head && (r->sigma_s != head->sigma_s || r->sigma_r != head->sigma_r ||
                         r->key.iters != head->key.iters || r->key.storage != head->key.storage)) {
                ++idx;
                continue;
            }
            Slot* sl = take_idle(s, r->key);
            if (!sl) {
                std::vector<Slot*> victims;
                const size_t need = shape_charge(r->key);
                if (!reserve(s, need, victims)) break;          // wait for room, in order
                s->queue.erase(s->queue.begin() + (long)idx);
                r->state = Request::RUNNING;
                lk.unlock();                                    // frees and allocations
                for (Slot* v : victims) destroy_slot(v);
                zncc_status st = ZNCC_OK;
                char err[256];
                sl = create_slot(r->key, need, &st, err, sizeof(err));
                lk.lock();
                if (!sl) {                                      // cannot run: fail it, go on
                    s->charged -= need;
                    snprintf(s->err, sizeof(s->err), "%s", err);
                    finish(s, r, st);
                    s->cv.notify_all();
                    continue;
                }
                s->slots.push_back(sl);
            } else {
                s->queue.erase(s->queue.begin() + (long)idx);
            }
            r->slot = sl;
            r->state = Request::RUNNING;
            b->reqs.push_back(r);
            if (!head) head = r;
            if (alone) break;
        }
        if (b->reqs.empty()) {
            delete b;
            continue;                                 // wait for a completion to free room
        }
        s->inflight += (int)b->reqs.size();
        seen = ~s->completions;                       // more may fit at once: look again
        lk.unlock();
        launch(s, b);
        lk.lock();
    }
    s->thread_done = true;
    s->cv.notify_all();
}

zncc_status check_request(int W, int H, int D, int win, float ss, float sr, int iters, int storage) {
    if (W < 1 || H < 1 || D < 1 || win < 3 || win > 15 || win % 2 == 0) return ZNCC_EINVAL;
    if (!(ss > 0.0f) || !(sr > 0.0f) || iters < 0 || iters > 64) return ZNCC_EINVAL;
    if (storage != ZNCC_F32 && storage != ZNCC_F16 && storage != ZNCC_I8) return ZNCC_EINVAL;
    if (W > 3072 || H > 4096 || D > 1024) return ZNCC_EUNSUPPORTED;
    return ZNCC_OK;
}

// Drops a request's share of its batch's timing; the last one returns the events to the pool.
// Under the lock.
void release_timing(zncc_server* s, Request* r) {
    BatchTiming* bt = r->timing;
    r->timing = nullptr;
    if (!bt || --bt->refs > 0) return;
    for (cudaEvent_t e : bt->ev)
        if (e) s->free_events.push_back(e);
    delete bt;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

extern "C" {

zncc_status serve_create(size_t volume_budget_bytes, int max_slots, zncc_server** out) {
    if (!out) return ZNCC_EINVAL;
    *out = nullptr;
    if (volume_budget_bytes == 0 || max_slots < 1) return ZNCC_EINVAL;
    zncc_server* s = new (std::nothrow) zncc_server();
    if (!s) return ZNCC_ENOMEM;
    s->budget = volume_budget_bytes;
    s->max_slots = max_slots;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        s->device = 0;
    }
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        delete s;
        return ZNCC_ENOMEM;
    }
    *out = s;
    return ZNCC_OK;
}

zncc_status serve_submit(zncc_server* s, const uint8_t* left_host, const uint8_t* right_host, int width,
                         int height, int max_disp, int win, float sigma_s, float sigma_r, int iters,
                         zncc_dtype storage, uint64_t* ticket) {
    if (!s || !left_host || !right_host || !ticket) return ZNCC_EINVAL;
    *ticket = 0;
    zncc_status st = check_request(width, height, max_disp, win, sigma_s, sigma_r, iters, storage);
    if (st != ZNCC_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        set_err(s, "serve_submit: %s", st == ZNCC_EINVAL ? "an argument is out of range"
                                                        : "a size beyond the kernels' limits");
        return st;
    }
    ShapeKey key{width, height, max_disp, win, (int)storage, iters};
    if (shape_charge(key) > s->budget) {                        // could never be admitted
        std::lock_guard<std::mutex> lk(s->mu);
        snprintf(s->err, sizeof(s->err), "serve_submit: the request needs %zu bytes of device memory, "
                 "more than the budget of %zu", shape_charge(key), s->budget);
        return ZNCC_EINVAL;
    }
    const size_t npix = (size_t)width * height;
    Request* r = new (std::nothrow) Request();
    if (!r) return ZNCC_ENOMEM;
    r->key = key;
    r->sigma_s = sigma_s;
    r->sigma_r = sigma_r;
    r->t_submit = Clock::now();
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stopping || s->tickets.size() >= kMaxQueued) {
        delete r;
        return ZNCC_EBUSY;
    }
    r->img = pool_take(s, 2 * npix);
    r->disp = pool_take(s, npix * sizeof(uint16_t));
    r->ticket = s->next_ticket++;
    lk.unlock();                                                // copies outside the lock
    if (!r->img.p) r->img = new_buf(2 * npix);
    if (!r->disp.p) r->disp = new_buf(npix * sizeof(uint16_t));
    if (!r->img.p || !r->disp.p) {
        drop_buf(r->img);
        drop_buf(r->disp);
        delete r;
        return ZNCC_ENOMEM;
    }
    memcpy(r->img.p, left_host, npix);                          // inputs copied before return
    memcpy(static_cast<uint8_t*>(r->img.p) + npix, right_host, npix);
    lk.lock();
    if (s->stopping) {
        give_buf(s, r->img);
        give_buf(s, r->disp);
        delete r;
        return ZNCC_EBUSY;
    }
    s->tickets[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
    lk.unlock();
    s->cv.notify_all();
    return ZNCC_OK;
}

zncc_status serve_poll(zncc_server* s, uint64_t ticket, uint16_t* disp_host, int timeout_us) {
    return serve_poll_timed(s, ticket, disp_host, timeout_us, nullptr);
}

zncc_status serve_poll_timed(zncc_server* s, uint64_t ticket, uint16_t* disp_host, int timeout_us,
                             zncc_serve_timing* timing) {
    if (!s || !disp_host || timeout_us < 0) return ZNCC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return ZNCC_EINVAL;
    Request* r = it->second;
    if (r->state != Request::DONE && timeout_us > 0)
        s->cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->state == Request::DONE; });
    if (r->state != Request::DONE) return timeout_us == 0 ? ZNCC_ENOTREADY : ZNCC_ETIMEOUT;
    const zncc_status st = r->status;
    if (st == ZNCC_OK) memcpy(disp_host, r->disp.p, (size_t)r->key.W * r->key.H * sizeof(uint16_t));
    if (timing) {
        *timing = zncc_serve_timing{};
        const BatchTiming* bt = r->timing;
        float e[3] = {0.f, 0.f, 0.f};
        // the events completed before the completion function ran, so these do not wait
        bool ok = st == ZNCC_OK && bt && bt->recorded;
        for (int k = 0; ok && k < 3; ++k) ok = cudaEventElapsedTime(&e[k], bt->ev[k], bt->ev[k + 1]) == cudaSuccess;
        if (!ok) cudaGetLastError();
        if (ok) {
            timing->queue_ms = ms_between(r->t_submit, r->t_issue);
            timing->h2d_ms = e[0];
            timing->run_ms = e[1];
            timing->d2h_ms = e[2];
            timing->total_ms = ms_between(r->t_submit, r->t_done);
            timing->device_wait_ms = timing->total_ms - timing->queue_ms - (e[0] + e[1] + e[2]);
            timing->batch_pairs = bt->pairs;
            timing->valid = 1;
        }
    }
    release_timing(s, r);
    s->tickets.erase(it);
    give_buf(s, r->img);
    give_buf(s, r->disp);
    delete r;
    return st;
}

zncc_status serve_destroy(zncc_server* s) {
    if (!s) return ZNCC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->stopping = true;
    for (Request* r : s->queue) finish(s, r, ZNCC_EBUSY);      // never started
    s->queue.clear();
    s->cv.notify_all();
    const auto deadline = Clock::now() + std::chrono::duration<double>(kDrainSeconds);
    const bool drained = s->cv.wait_until(lk, deadline, [&] { return s->thread_done && s->inflight == 0; });
    if (!drained) {
        // In-flight GPU work did not finish in time: its buffers cannot be freed safely.
        // The server stays allocated (leaked) and the scheduler thread is left to end.
        set_err(s, "serve_destroy: in-flight work did not finish within the drain limit");
        lk.unlock();
        s->worker.detach();
        return ZNCC_ETIMEOUT;
    }
    lk.unlock();
    s->worker.join();
    for (Slot* sl : s->slots) destroy_slot(sl);
    for (auto& kv : s->tickets) {
        release_timing(s, kv.second);
        drop_buf(kv.second->img);
        drop_buf(kv.second->disp);
        delete kv.second;
    }
    for (auto& kv : s->free_bufs) drop_buf(kv.second);
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    for (cudaStream_t st : s->streams)
        if (st) cudaStreamDestroy(st);
    delete s;
    return ZNCC_OK;
}

const char* serve_last_error(const zncc_server* s) { return s ? s->err : ""; }

}  // extern "C"
