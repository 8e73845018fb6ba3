// Serving engine: continuous batching of decode + Compass requests under a
// fixed device-memory budget (the multi-stream host framework the paper
// runs in, Sec. I, made a request loop).
//
// A request is one batch of events (host buffers: raw banks, event offsets,
// VELO tracks) plus host output buffers for its track slots.  The engine
// owns one device arena of `budget` bytes and `n_slots` streams.  A worker
// thread admits waiting requests in arrival order as soon as a slot is idle
// and the arena can hold the request's buffers; an admitted request's
// copies in, its single batched launch (ut_run_batched) and its copies out
// are enqueued on the slot's stream -- outside the engine's lock, so that
// submissions and polls never wait behind an enqueue -- and requests overlap
// on the device.  A host function enqueued after the copies out marks the
// request complete as soon as the stream reaches it (no polling): the
// request's arena block is freed, its latency (submission to completion,
// host clock) recorded and the worker woken for the next admissions.

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace utc {

using Clock = std::chrono::steady_clock;

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit allocator over [0, size) with coalescing frees.
class Arena {
   public:
    explicit Arena(size_t size) { free_[0] = size; }
    bool alloc(size_t n, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n;
                const size_t start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

   private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct Request {
    int64_t id;
    ut_server_request in;
    size_t bytes = 0, off = 0;
    int slot = -1;
    Clock::time_point t_submit, t_admit, t_done;
    int status = UT_OK;
    int64_t where_a = -1, where_b = -1;
};

struct Slot {
    cudaStream_t stream = nullptr;
    ut_ctx* ctx = nullptr;
    Request* req = nullptr;
    ut_server* sv = nullptr;
};

}  // namespace utc

struct ut_server {
    ut_geometry geom;
    compass_params params;
    ut_launch_config cfg;
    size_t budget = 0;
    char* d_arena = nullptr;
    utc::Arena* arena = nullptr;
    std::vector<utc::Slot> slots;
    std::deque<utc::Request*> pending;
    std::vector<utc::Request*> finished;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    int64_t next_id = 0;
    int64_t in_flight = 0;
    int device = 0;
    size_t peak_used = 0;
};

namespace utc {

// Device layout of one request inside its arena block.
struct Layout {
    size_t raw, ev_off, vx, vy, vtx, vty, flags, trk_off, x, z, sector, layer, id, hit_off;
    size_t hit, qop, chi2, ox, otx, nhits, found, ws, total;
    uint32_t capacity;
};

static Layout layout_of(const ut_server_request& r, int S) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t n) {
        const size_t at = o;
        o += align256(n);
        return at;
    };
    const size_t T = r.n_tracks, E = (size_t)r.n_events, B = (size_t)4 * S;
    const size_t words = (r.n_raw_words + 3) / 4 * 4;
    const size_t cap = 2 * (size_t)r.n_raw_words + 1;
    L.capacity = (uint32_t)std::min<size_t>(cap, 0xFFFFFFFFu);
    L.raw = take(words * 4);
    L.ev_off = take((E + 1) * 8);
    L.vx = take(T * 4);
    L.vy = take(T * 4);
    L.vtx = take(T * 4);
    L.vty = take(T * 4);
    L.flags = take(T);
    L.trk_off = take((E + 1) * 4);
    L.x = take(cap * 4);
    L.z = take(cap * 4);
    L.sector = take(cap * 2);
    L.layer = take(cap);
    L.id = take(cap * 4);
    L.hit_off = take((E * B + 1) * 4);
    L.hit = take(T * 16);
    L.qop = take(T * 4);
    L.chi2 = take(T * 4);
    L.ox = take(T * 4);
    L.otx = take(T * 4);
    L.nhits = take(T);
    L.found = take(T);
    L.ws = take(ut_decode_workspace_size((int)E));
    L.total = o;
    return L;
}

static void set_error(Request* q, int rc) {
    if (q->status == UT_OK) q->status = rc;
}

// Enqueue one admitted request's copies, launch and copies out on its slot's
// stream (called without the engine's lock: the slot and the arena block
// belong to this request until it completes; only enqueues work).
static void launch_request(ut_server* sv, Slot& sl, Request* q) {
    const ut_server_request& r = q->in;
    const Layout L = layout_of(r, sv->geom.n_sectors);
    char* base = sv->d_arena + q->off;
    cudaStream_t st = sl.stream;
    const size_t T = r.n_tracks, E = (size_t)r.n_events;
    auto h2d = [&](size_t off, const void* src, size_t n) {
        if (n && cudaMemcpyAsync(base + off, src, n, cudaMemcpyHostToDevice, st) != cudaSuccess)
            set_error(q, UT_ERR_CUDA);
    };
    auto d2h = [&](void* dst, size_t off, size_t n) {
        if (n && dst && cudaMemcpyAsync(dst, base + off, n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            set_error(q, UT_ERR_CUDA);
    };
    h2d(L.raw, r.raw, r.n_raw_words * 4);
    h2d(L.ev_off, r.ev_off, (E + 1) * 8);
    h2d(L.vx, r.vx, T * 4);
    h2d(L.vy, r.vy, T * 4);
    h2d(L.vtx, r.vtx, T * 4);
    h2d(L.vty, r.vty, T * 4);
    h2d(L.flags, r.flags, T);
    h2d(L.trk_off, r.trk_off, (E + 1) * 4);
    ut_hits hits;
    hits.x = reinterpret_cast<float*>(base + L.x);
    hits.z = reinterpret_cast<float*>(base + L.z);
    hits.sector = reinterpret_cast<uint16_t*>(base + L.sector);
    hits.layer = reinterpret_cast<uint8_t*>(base + L.layer);
    hits.id = reinterpret_cast<uint32_t*>(base + L.id);
    hits.hit_off = reinterpret_cast<uint32_t*>(base + L.hit_off);
    hits.capacity = L.capacity;
    velo_tracks velo;
    velo.x = reinterpret_cast<const float*>(base + L.vx);
    velo.y = reinterpret_cast<const float*>(base + L.vy);
    velo.tx = reinterpret_cast<const float*>(base + L.vtx);
    velo.ty = reinterpret_cast<const float*>(base + L.vty);
    velo.flags = reinterpret_cast<const uint8_t*>(base + L.flags);
    velo.trk_off = reinterpret_cast<const uint32_t*>(base + L.trk_off);
    compass_tracks tr{};
    tr.hit = reinterpret_cast<int32_t*>(base + L.hit);
    tr.qop = reinterpret_cast<float*>(base + L.qop);
    tr.chi2 = reinterpret_cast<float*>(base + L.chi2);
    tr.x = reinterpret_cast<float*>(base + L.ox);
    tr.tx = reinterpret_cast<float*>(base + L.otx);
    tr.nhits = reinterpret_cast<uint8_t*>(base + L.nhits);
    tr.found = reinterpret_cast<uint8_t*>(base + L.found);
    if (cudaMemsetAsync(sl.ctx->d_status, 0xFF, sizeof(unsigned long long), st) != cudaSuccess)
        set_error(q, UT_ERR_CUDA);
    if (q->status == UT_OK) {
        const int rc = ut_run_batched(sl.ctx, reinterpret_cast<const uint32_t*>(base + L.raw), r.n_raw_words,
                                      reinterpret_cast<const uint64_t*>(base + L.ev_off), r.n_events, &velo,
                                      r.n_tracks, &sv->params, &hits, &tr, &sv->cfg, base + L.ws,
                                      ut_decode_workspace_size(r.n_events), st);
        if (rc != UT_OK) set_error(q, rc);
    }
    d2h(r.out_hit, L.hit, T * 16);
    d2h(r.out_qop, L.qop, T * 4);
    d2h(r.out_chi2, L.chi2, T * 4);
    d2h(r.out_x, L.ox, T * 4);
    d2h(r.out_tx, L.otx, T * 4);
    d2h(r.out_nhits, L.nhits, T);
    d2h(r.out_found, L.found, T);
    if (cudaMemcpyAsync(sl.ctx->h_status, sl.ctx->d_status, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess)
        set_error(q, UT_ERR_CUDA);
}

// Completion of a slot's request, with the engine's lock held: the status
// word (copied to page-locked memory before the host function ran), the
// arena block freed, the result queued for ut_server_poll.
static void finish_request(ut_server* sv, Slot& sl) {
    Request* r = sl.req;
    r->t_done = Clock::now();
    const unsigned long long k = *sl.ctx->h_status;
    if (k != ~0ull && r->status == UT_OK) {
        r->status = -(int)(k & 0xFF);
        const unsigned long long a = k >> 32, b = (k >> 8) & 0xFFFFFF;
        r->where_a = a == 0xFFFFFFFFull ? -1 : (int64_t)a;
        r->where_b = b == 0xFFFFFFull ? -1 : (int64_t)b;
    }
    sv->arena->release(r->off, r->bytes);
    sl.req = nullptr;
    sv->finished.push_back(r);
    --sv->in_flight;
}

// Host function enqueued after a request's copies out: runs on a CUDA
// driver thread once the stream has reached it (it makes no CUDA call).
static void CUDART_CB on_request_done(void* user) {
    Slot* sl = static_cast<Slot*>(user);
    ut_server* sv = sl->sv;
    std::lock_guard<std::mutex> lk(sv->mu);
    finish_request(sv, *sl);
    sv->cv.notify_all();
}

static void worker_loop(ut_server* sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    std::vector<Slot*> admitted;
    while (true) {
        // admissions, in arrival order, while a slot and memory are free
        admitted.clear();
        while (!sv->pending.empty()) {
            Request* r = sv->pending.front();
            Slot* free_slot = nullptr;
            for (Slot& sl : sv->slots)
                if (!sl.req) {
                    free_slot = &sl;
                    break;
                }
            if (!free_slot) break;
            size_t off = 0;
            if (!sv->arena->alloc(r->bytes, &off)) break;
            sv->pending.pop_front();
            r->off = off;
            r->t_admit = Clock::now();
            r->slot = (int)(free_slot - sv->slots.data());
            free_slot->req = r;
            sv->peak_used = std::max(sv->peak_used, sv->arena->used());
            admitted.push_back(free_slot);
        }
        if (!admitted.empty()) {
            // enqueue outside the lock; the slots stay owned by their requests
            lk.unlock();
            for (Slot* sl : admitted) {
                launch_request(sv, *sl, sl->req);
                if (cudaLaunchHostFunc(sl->stream, on_request_done, sl) != cudaSuccess) {
                    cudaStreamSynchronize(sl->stream);  // the request can still be finished here
                    std::lock_guard<std::mutex> g(sv->mu);
                    set_error(sl->req, UT_ERR_CUDA);
                    finish_request(sv, *sl);
                    sv->cv.notify_all();
                }
            }
            lk.lock();
            continue;
        }
        if (sv->stop && sv->pending.empty() && sv->in_flight == 0) break;
        // wait for a submission or a completion (both notify)
        sv->cv.wait(lk);
    }
}

}  // namespace utc

using namespace utc;

extern "C" size_t ut_server_request_bytes(const ut_geometry* geom, const ut_server_request* r) {
    if (!geom || !r) return 0;
    return layout_of(*r, geom->n_sectors).total;
}

extern "C" int ut_server_create(ut_server** out, const ut_geometry* geom, const compass_params* p,
                                size_t budget_bytes, int n_slots, const ut_launch_config* cfg) {
    if (!out || !geom || !p || n_slots < 1 || n_slots > 64 || budget_bytes < 4096) return UT_ERR_ARG;
    if (p->output_order != 0) return UT_ERR_ARG;  // request outputs are per VELO slot
    *out = nullptr;
    ut_server* sv = new (std::nothrow) ut_server();
    if (!sv) return UT_ERR_ARG;
    sv->geom = *geom;
    sv->params = *p;
    sv->cfg = cfg ? *cfg : ut_launch_config{0, 0, 0, 0};
    sv->budget = budget_bytes & ~(size_t)255;
    if (cudaGetDevice(&sv->device) != cudaSuccess || cudaMalloc(&sv->d_arena, sv->budget) != cudaSuccess) {
        delete sv;
        return UT_ERR_CUDA;
    }
    sv->arena = new Arena(sv->budget);
    sv->slots.resize(n_slots);
    for (Slot& sl : sv->slots) {
        sl.sv = sv;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            ut_ctx_create(&sl.ctx, geom) != UT_OK) {
            ut_server_destroy(sv);
            return UT_ERR_CUDA;
        }
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return UT_OK;
}

extern "C" int64_t ut_server_submit(ut_server* sv, const ut_server_request* r) {
    if (!sv || !r || r->n_events < 1 || !r->raw || !r->ev_off || !r->trk_off) return UT_ERR_ARG;
    if (r->n_tracks > 0 && (!r->vx || !r->vy || !r->vtx || !r->vty || !r->flags)) return UT_ERR_ARG;
    Request* q = new (std::nothrow) Request();
    if (!q) return UT_ERR_ARG;
    q->in = *r;
    q->bytes = layout_of(*r, sv->geom.n_sectors).total;
    if (q->bytes > sv->budget) {
        delete q;
        return UT_ERR_CAPACITY;
    }
    q->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    q->id = sv->next_id++;
    sv->pending.push_back(q);
    ++sv->in_flight;
    sv->cv.notify_all();
    return q->id;
}

extern "C" int ut_server_poll(ut_server* sv, ut_server_result* results, int max_results, int wait) {
    if (!sv || (!results && max_results > 0) || max_results < 0) return UT_ERR_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (wait && sv->finished.empty() && sv->in_flight > 0)
        sv->cv.wait(lk, [&] { return !sv->finished.empty() || sv->in_flight == 0; });
    const int n = std::min<int>(max_results, (int)sv->finished.size());
    for (int i = 0; i < n; ++i) {
        Request* q = sv->finished[i];
        ut_server_result& o = results[i];
        o.id = q->id;
        o.status = q->status;
        o.where_a = q->where_a;
        o.where_b = q->where_b;
        o.queue_s = std::chrono::duration<double>(q->t_admit - q->t_submit).count();
        o.latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
        o.slot = q->slot;
        delete q;
    }
    sv->finished.erase(sv->finished.begin(), sv->finished.begin() + n);
    return n;
}

extern "C" int ut_server_stats(ut_server* sv, int64_t* in_flight, size_t* arena_used, size_t* arena_peak) {
    if (!sv) return UT_ERR_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (in_flight) *in_flight = sv->in_flight;
    if (arena_used) *arena_used = sv->arena->used();
    if (arena_peak) *arena_peak = sv->peak_used;
    return UT_OK;
}

extern "C" int ut_server_destroy(ut_server* sv) {
    if (!sv) return UT_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    for (Slot& sl : sv->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ctx) ut_ctx_destroy(sl.ctx);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (Request* q : sv->finished) delete q;
    cudaFree(sv->d_arena);
    delete sv->arena;
    delete sv;
    return UT_OK;
}
