// Serving loop: continuous batching of FFT requests under a device-memory budget.
//
// Requests (n, batch, direction, host input, host output) are submitted from
// any thread and queued with their arrival time.  One worker thread owns the
// device side:
//   admission   FIFO: the head request is admitted when its slot (8*n*batch
//               bytes of data, twice that for two-pass lengths) fits in what
//               is left of a device arena of `budget` bytes (first-fit
//               allocator over one cudaMalloc made at start-up); a request
//               larger than the whole budget is refused at submit time.
//   batching    the requests admitted in one round are grouped by
//               (n, direction); each group gets one contiguous slot, one
//               launch over all its rows and one stream out of a pool, so
//               requests that arrive while others are on the GPU are admitted
//               as memory frees up and their copies and kernels overlap the
//               earlier groups' work.
//   plans       per (n, direction) the schedule and its twiddle tables are
//               built once and stay resident.
//   completion  an event recorded after a group's device-to-host copies;
//               the worker polls it, stamps the completion time when it
//               finds it complete and frees the slot.  Latency = completion -
//               arrival.  (Host-function callbacks were used first; runs of
//               a few seconds then showed pauses of 40-120 ms in the device-
//               side service of a few hundred requests.)
// Serial mode (one stream, one request per group, one request in flight) is
// the naive queue the batching loop is compared with.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace gbfft {
namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0, Clock::time_point t) {
    return std::chrono::duration<double>(t - t0).count();
}

// First-fit allocator over [0, size) in 256-byte units.
class Arena {
  public:
    explicit Arena(size_t size) : size_(size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
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
    size_t used() const { return used_; }
    size_t size() const { return size_; }

  private:
    size_t size_, used_ = 0;
    std::map<size_t, size_t> free_;
};

struct ServerPlan {  // resident schedule for one (n, direction)
    bool two_pass = false;
    const RowsVariant* rv = nullptr;
    int grid_cap = 0;
    float2* tw = nullptr;
    int64_t k = 1, m = 0;
    const ColsVariant *cm = nullptr, *ck = nullptr;
    float2 *tw_m = nullptr, *tw_k = nullptr, *post = nullptr;
};

enum ReqState : int { kQueued = 0, kRunning = 1, kDone = 2, kCancelled = 3, kFailed = 4 };

struct Request {
    uint64_t ticket;
    int64_t n, batch;
    int direction;
    const void* in;
    void* out;
    Clock::time_point arrival, admitted;
    double latency = 0;
    double queued = 0;  // admitted - arrival: waiting in the server queue
    int state = kQueued;
};

struct Group {
    std::vector<Request*> reqs;
    size_t off = 0, bytes = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;  // recorded after the group's copies back
    Clock::time_point completed;
};

}  // namespace

constexpr size_t kWarmScratchBytes = size_t(4) << 20;  // one row (and its two-pass workspace) up to N = 262144

struct Server {
    int device = 0;
    float2* scratch = nullptr;  // kWarmScratchBytes, for the warm-up launch of each new plan
    size_t budget = 0;
    bool serial = false;
    char* arena_base = nullptr;
    std::unique_ptr<Arena> arena;
    std::vector<cudaStream_t> streams;
    cudaStream_t tstream = nullptr;  // plan tables are built here, off the serving streams
    int* status = nullptr;           // device status word for bounded waits of the kernels
    int next_stream = 0;
    std::map<std::pair<int64_t, int>, ServerPlan> plans;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> table;
    std::vector<std::unique_ptr<Group>> inflight;
    std::vector<cudaEvent_t> free_events, all_events;  // completion events, reused
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    int error = GBFFT_OK;

    // statistics (under mu)
    std::vector<double> latencies;
    Clock::time_point win_start = Clock::now(), win_last = Clock::now();
    double bytes_done = 0;
    size_t groups_launched = 0, max_inflight_reqs = 0, max_used = 0;
};

namespace {

gbfft_status get_plan(Server* s, int64_t n, int dir, ServerPlan** out) {
    auto key = std::make_pair(n, dir);
    auto it = s->plans.find(key);
    if (it != s->plans.end()) {
        *out = &it->second;
        return GBFFT_OK;
    }
    ServerPlan sp;
    const RowsVariant* cands[1];
    if (rows_variants_for(n, cands, 1) > 0) {
        sp.rv = cands[0];
        if (prepare_rows(*sp.rv) != cudaSuccess) return GBFFT_ERR_CUDA;
        if (sp.rv->kind == kRowsPersistent || sp.rv->kind == kRowsTma) sp.grid_cap = persistent_grid(*sp.rv);
        const int cnt = stage_twiddle_count(sp.rv->radix, sp.rv->nstages);
        if (cudaMalloc(&sp.tw, sizeof(float2) * (size_t)std::max(cnt, 1)) != cudaSuccess) return GBFFT_ERR_OOM;
        if (launch_stage_twiddles(sp.tw, n, sp.rv->radix, sp.rv->nstages, s->tstream) != cudaSuccess) return GBFFT_ERR_CUDA;
    } else {
        if (!choose_split(n, 0, &sp.k, &sp.m)) return GBFFT_ERR_UNSUPPORTED_SIZE;
        sp.two_pass = true;
        sp.cm = cols_variant_for(sp.m);
        sp.ck = cols_variant_for(sp.k);
        if (prepare_cols(*sp.cm) != cudaSuccess || prepare_cols(*sp.ck) != cudaSuccess) return GBFFT_ERR_CUDA;
        const int cm_cnt = stage_twiddle_count(sp.cm->radix, sp.cm->nstages);
        const int ck_cnt = stage_twiddle_count(sp.ck->radix, sp.ck->nstages);
        if (cudaMalloc(&sp.tw_m, sizeof(float2) * (size_t)std::max(cm_cnt, 1)) != cudaSuccess ||
            cudaMalloc(&sp.tw_k, sizeof(float2) * (size_t)std::max(ck_cnt, 1)) != cudaSuccess ||
            cudaMalloc(&sp.post, sizeof(float2) * (size_t)n) != cudaSuccess)
            return GBFFT_ERR_OOM;
        if (launch_stage_twiddles(sp.tw_m, sp.m, sp.cm->radix, sp.cm->nstages, s->tstream) != cudaSuccess ||
            launch_stage_twiddles(sp.tw_k, sp.k, sp.ck->radix, sp.ck->nstages, s->tstream) != cudaSuccess ||
            launch_post_twiddles(sp.post, n, sp.m, s->tstream) != cudaSuccess)
            return GBFFT_ERR_CUDA;
    }
    // Run the plan once on one row of the server's own scratch buffer: the first launch of a kernel
    // loads its module, which must not happen inside a request's latency.
    if ((size_t)n * 2 * sizeof(float2) <= kWarmScratchBytes) {
        float2* scratch = s->scratch;
        if (!sp.two_pass) {
            if (launch_rows(*sp.rv, dir, scratch, scratch, sp.tw, 1, sp.grid_cap, s->tstream, s->status) != cudaSuccess)
                return GBFFT_ERR_CUDA;
        } else {
            float2* ws = scratch + n;
            if (launch_cols(*sp.cm, 1, dir, scratch, ws, sp.tw_m, sp.post, 1, (int)sp.k, s->tstream) != cudaSuccess ||
                launch_cols(*sp.ck, 2, dir, ws, scratch, sp.tw_k, nullptr, 1, (int)sp.m, s->tstream) != cudaSuccess)
                return GBFFT_ERR_CUDA;
        }
    }
    if (cudaStreamSynchronize(s->tstream) != cudaSuccess) return GBFFT_ERR_CUDA;
    auto res = s->plans.emplace(key, sp);
    *out = &res.first->second;
    return GBFFT_OK;
}

size_t slot_bytes(int64_t n, int64_t rows, bool two_pass) {
    const size_t b = sizeof(float2) * (size_t)n * (size_t)rows;
    return two_pass ? 2 * ((b + 255) & ~size_t(255)) : b;
}

bool needs_two_pass(int64_t n) { return rows_variants_for(n, nullptr, 0) == 0; }

// Launch one group: H2D of each request into the slot, one transform over
// all rows (in place), D2H of each request, completion stamp.
bool launch_group(Server* s, Group* g, ServerPlan* sp, int64_t n, int dir, int64_t rows) {
    float2* data = (float2*)(s->arena_base + g->off);
    const size_t row_bytes = sizeof(float2) * (size_t)n;
    bool ok = true;
    size_t at = 0;
    for (Request* r : g->reqs) {
        ok = ok && cudaMemcpyAsync((char*)data + at, r->in, row_bytes * (size_t)r->batch, cudaMemcpyHostToDevice,
                                   g->stream) == cudaSuccess;
        at += row_bytes * (size_t)r->batch;
    }
    if (!sp->two_pass) {
        ok = ok && launch_rows(*sp->rv, dir, data, data, sp->tw, (long long)rows, sp->grid_cap, g->stream,
                               s->status) == cudaSuccess;
    } else {
        float2* ws = (float2*)((char*)data + ((row_bytes * (size_t)rows + 255) & ~size_t(255)));
        ok = ok && launch_cols(*sp->cm, 1, dir, data, ws, sp->tw_m, sp->post, (long long)rows, (int)sp->k,
                               g->stream) == cudaSuccess;
        ok = ok && launch_cols(*sp->ck, 2, dir, ws, data, sp->tw_k, nullptr, (long long)rows, (int)sp->m,
                               g->stream) == cudaSuccess;
    }
    at = 0;
    for (Request* r : g->reqs) {
        ok = ok && cudaMemcpyAsync(r->out, (char*)data + at, row_bytes * (size_t)r->batch, cudaMemcpyDeviceToHost,
                                   g->stream) == cudaSuccess;
        at += row_bytes * (size_t)r->batch;
    }
    ok = ok && cudaEventRecord(g->ev, g->stream) == cudaSuccess;
    return ok;
}

void worker_main(Server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // 1. retire finished groups.  A stream runs its groups in launch order, so only the oldest
        //    unfinished group of each stream is queried: at most one pending query per stream,
        //    however many groups are in flight.
        {
            std::vector<cudaStream_t> pending;
            size_t keep = 0;
            for (size_t i = 0; i < s->inflight.size(); ++i) {
                Group* g = s->inflight[i].get();
                const bool blocked = std::find(pending.begin(), pending.end(), g->stream) != pending.end();
                if (blocked || cudaEventQuery(g->ev) != cudaSuccess) {
                    if (!blocked) pending.push_back(g->stream);
                    if (keep != i) s->inflight[keep] = std::move(s->inflight[i]);
                    ++keep;
                    continue;
                }
                g->completed = Clock::now();
                s->free_events.push_back(g->ev);
                for (Request* r : g->reqs) {
                    r->latency = seconds_since(r->arrival, g->completed);
                    r->queued = seconds_since(r->arrival, r->admitted);
                    r->state = kDone;
                    s->latencies.push_back(r->latency);
                    s->bytes_done += 16.0 * (double)r->n * (double)r->batch;
                }
                s->win_last = g->completed;
                s->arena->release(g->off, g->bytes);
                s->inflight[i].reset();
                s->cv.notify_all();
            }
            s->inflight.resize(keep);
        }
        if (s->stop && s->queue.empty() && s->inflight.empty()) break;
        // 2. admit from the head of the queue while slots fit
        std::vector<Request*> admitted;
        size_t inflight_reqs = 0;
        for (auto& g : s->inflight) inflight_reqs += g->reqs.size();
        std::map<std::pair<int64_t, int>, std::vector<Request*>> groups;
        size_t pending_bytes = 0;
        while (!s->queue.empty()) {
            if (s->serial && (inflight_reqs + admitted.size()) >= 1) break;
            Request* r = s->queue.front();
            const size_t need = slot_bytes(r->n, r->batch, needs_two_pass(r->n)) + 256;
            if (s->arena->used() + pending_bytes + need > s->arena->size()) break;
            s->queue.pop_front();
            admitted.push_back(r);
            pending_bytes += need;
            groups[{r->n, r->direction}].push_back(r);
        }
        // 3. one slot, one launch per (n, direction) group; a group whose slot
        //    does not fit contiguously (fragmentation) is retried request by
        //    request, and what still does not fit returns to the queue front.
        std::vector<Request*> retry;
        auto start_group = [&](std::vector<Request*> reqs, int64_t n, int dir, ServerPlan* sp) -> bool {
            int64_t rows = 0;
            for (Request* r : reqs) rows += r->batch;
            auto g = std::make_unique<Group>();
            g->reqs = std::move(reqs);
            g->bytes = slot_bytes(n, rows, sp->two_pass);
            if (!s->arena->alloc(g->bytes, &g->off)) return false;
            if (s->free_events.empty()) {
                cudaEvent_t ev;
                if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
                    s->arena->release(g->off, g->bytes);
                    return false;
                }
                s->all_events.push_back(ev);
                s->free_events.push_back(ev);
            }
            g->ev = s->free_events.back();
            s->free_events.pop_back();
            g->stream = s->streams[(size_t)s->next_stream];
            s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
            const Clock::time_point now = Clock::now();
            for (Request* r : g->reqs) {
                r->state = kRunning;
                r->admitted = now;
            }
            // The copies and launches run without the lock: the group's requests are Running (no other
            // thread changes or releases them), its slot and event are the worker's, and submissions
            // need not wait behind a group's API calls.
            lk.unlock();
            const bool launched = launch_group(s, g.get(), sp, n, dir, rows);
            lk.lock();
            if (!launched) {
                s->error = GBFFT_ERR_CUDA;
                for (Request* r : g->reqs) r->state = kFailed;
                cudaStreamSynchronize(g->stream);
                s->free_events.push_back(g->ev);
                s->arena->release(g->off, g->bytes);
                s->cv.notify_all();
                return true;
            }
            ++s->groups_launched;
            s->inflight.push_back(std::move(g));
            return true;
        };
        for (auto& kv : groups) {
            const int64_t n = kv.first.first;
            const int dir = kv.first.second;
            ServerPlan* sp = nullptr;
            const gbfft_status st = get_plan(s, n, dir, &sp);
            if (st != GBFFT_OK) {
                s->error = st;
                for (Request* r : kv.second) r->state = kFailed;
                s->cv.notify_all();
                continue;
            }
            if (start_group(kv.second, n, dir, sp)) continue;
            for (Request* r : kv.second)
                if (!start_group({r}, n, dir, sp)) retry.push_back(r);
        }
        if (!retry.empty()) {
            std::sort(retry.begin(), retry.end(), [](const Request* a, const Request* b) { return a->ticket < b->ticket; });
            for (auto it = retry.rbegin(); it != retry.rend(); ++it) s->queue.push_front(*it);
        }
        inflight_reqs = 0;
        for (auto& g : s->inflight) inflight_reqs += g->reqs.size();
        s->max_inflight_reqs = std::max(s->max_inflight_reqs, inflight_reqs);
        s->max_used = std::max(s->max_used, s->arena->used());
        // 4. idle: sleep on the condition variable; with groups in flight, yield and poll again.
        //    (A loop that polled the events without the lock and woke on every submission launched
        //    one small group per arrival and measured a worse tail.)
        if (s->inflight.empty() && s->queue.empty() && !s->stop) {
            s->cv.wait_for(lk, std::chrono::milliseconds(5));
        } else {
            lk.unlock();
            std::this_thread::yield();  // completions are observed by polling their events
            lk.lock();
        }
    }
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = p * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

}  // namespace

gbfft_status server_create(Server** out, size_t budget, int n_streams, int flags) {
    *out = nullptr;
    if (budget < (size_t(1) << 20) || n_streams < 1 || n_streams > 64) return GBFFT_ERR_INVALID_ARG;
    Server* s = new (std::nothrow) Server();
    if (!s) return GBFFT_ERR_OOM;
    s->serial = (flags & 1) != 0;
    if (s->serial) n_streams = 1;
    s->budget = budget;
    if (cudaGetDevice(&s->device) != cudaSuccess || cudaMalloc(&s->arena_base, budget) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return GBFFT_ERR_OOM;
    }
    s->arena.reset(new Arena(budget));
    if (cudaMalloc(&s->status, sizeof(int)) != cudaSuccess || cudaMemset(s->status, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&s->scratch, kWarmScratchBytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->arena_base);
        delete s;
        return GBFFT_ERR_OOM;
    }
    if (cudaStreamCreateWithFlags(&s->tstream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(s->arena_base);
        delete s;
        return GBFFT_ERR_CUDA;
    }
    for (int i = 0; i < n_streams; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            cudaFree(s->arena_base);
            delete s;
            return GBFFT_ERR_CUDA;
        }
        s->streams.push_back(st);
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return GBFFT_OK;
}

gbfft_status server_submit(Server* s, int64_t n, int64_t batch, int direction, const void* in, void* out,
                           uint64_t* ticket, const Clock::time_point* arrival = nullptr) {
    if (!s || !in || !out || !ticket || batch < 1 || n < 1) return GBFFT_ERR_INVALID_ARG;
    if (direction != GBFFT_FORWARD && direction != GBFFT_INVERSE) return GBFFT_ERR_INVALID_ARG;
    int64_t kk = 0, mm = 0;
    if (rows_variants_for(n, nullptr, 0) == 0 && !choose_split(n, 0, &kk, &mm)) return GBFFT_ERR_UNSUPPORTED_SIZE;
    if (slot_bytes(n, batch, needs_two_pass(n)) + 256 > s->budget) return GBFFT_ERR_BUDGET;
    auto r = std::make_unique<Request>();
    r->n = n;
    r->batch = batch;
    r->direction = direction;
    r->in = in;
    r->out = out;
    r->arrival = arrival ? *arrival : Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return GBFFT_ERR_INVALID_ARG;
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->table.emplace(r->ticket, std::move(r));
    s->cv.notify_all();
    return GBFFT_OK;
}

gbfft_status server_prepare(Server* s, int64_t n, int direction) {
    if (direction != GBFFT_FORWARD && direction != GBFFT_INVERSE) return GBFFT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    ServerPlan* sp = nullptr;
    return get_plan(s, n, direction, &sp);
}

gbfft_status server_poll(Server* s, uint64_t ticket, int* done, double* latency) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return GBFFT_ERR_NOT_FOUND;
    const Request* r = it->second.get();
    if (done) *done = r->state == kDone ? 1 : (r->state == kFailed || r->state == kCancelled ? -1 : 0);
    if (latency) *latency = r->latency;
    return r->state == kFailed ? (s->error ? (gbfft_status)s->error : GBFFT_ERR_CUDA) : GBFFT_OK;
}

gbfft_status server_timing(Server* s, uint64_t ticket, double* queued, double* latency) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return GBFFT_ERR_NOT_FOUND;
    const Request* r = it->second.get();
    if (r->state != kDone) return GBFFT_ERR_INVALID_ARG;
    if (queued) *queued = r->queued;
    if (latency) *latency = r->latency;
    return GBFFT_OK;
}

gbfft_status server_wait(Server* s, uint64_t ticket, double timeout_s) {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return GBFFT_ERR_NOT_FOUND;
    Request* r = it->second.get();
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s));
    while (r->state == kQueued || r->state == kRunning) {
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout &&
            (r->state == kQueued || r->state == kRunning))
            return GBFFT_ERR_TIMEOUT;
    }
    return r->state == kDone ? GBFFT_OK : GBFFT_ERR_CUDA;
}

gbfft_status server_release(Server* s, uint64_t ticket) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return GBFFT_ERR_NOT_FOUND;
    if (it->second->state == kQueued || it->second->state == kRunning) return GBFFT_ERR_INVALID_ARG;
    s->table.erase(it);
    return GBFFT_OK;
}

void server_stats(Server* s, double* out, int nout) {
    std::lock_guard<std::mutex> lk(s->mu);
    double v[10] = {0};
    v[0] = (double)s->latencies.size();
    v[1] = percentile(s->latencies, 0.50);
    v[2] = percentile(s->latencies, 0.99);
    v[3] = s->latencies.empty() ? 0.0 : *std::max_element(s->latencies.begin(), s->latencies.end());
    const double win = seconds_since(s->win_start, s->win_last);
    v[4] = win > 0 ? (double)s->latencies.size() / win : 0.0;
    v[5] = win > 0 ? s->bytes_done / win / 1e9 : 0.0;
    v[6] = (double)s->groups_launched;
    v[7] = (double)s->max_inflight_reqs;
    v[8] = (double)s->max_used;
    v[9] = win;
    for (int i = 0; i < nout && i < 10; ++i) out[i] = v[i];
}

void server_reset_stats(Server* s) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->latencies.clear();
    s->bytes_done = 0;
    s->groups_launched = 0;
    s->max_inflight_reqs = 0;
    s->max_used = 0;
    s->win_start = s->win_last = Clock::now();
}

// Submit requests at their arrival offsets (seconds after the call) from this
// thread: an open-loop generator, so a slow server does not delay arrivals.
gbfft_status server_replay(Server* s, int64_t count, const int64_t* n, const int64_t* batch, const int* direction,
                           const void* const* in, void* const* out, const double* arrival_s, uint64_t* tickets) {
    const Clock::time_point t0 = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->win_start = s->win_last = t0;
    }
    for (int64_t i = 0; i < count; ++i) {
        const Clock::time_point due =
            t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
        while (Clock::now() < due) {
            const auto left = due - Clock::now();
            if (left > std::chrono::microseconds(200)) std::this_thread::sleep_for(left - std::chrono::microseconds(100));
        }
        // latency counts from the scheduled arrival: a submission that runs late (the submitting
        // thread delayed) still owes the request its wait
        gbfft_status st = server_submit(s, n[i], batch[i], direction[i], in[i], out[i], &tickets[i], &due);
        if (st != GBFFT_OK) return st;
    }
    return GBFFT_OK;
}

void server_destroy(Server* s) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // queued requests that never started are cancelled
        for (Request* r : s->queue) r->state = kCancelled;
        s->queue.clear();
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    cudaStreamSynchronize(s->tstream);
    cudaStreamDestroy(s->tstream);
    for (auto& kv : s->plans) {
        ServerPlan& p = kv.second;
        float2* bufs[] = {p.tw, p.tw_m, p.tw_k, p.post};
        for (float2* b : bufs)
            if (b) cudaFree(b);
    }
    for (cudaEvent_t ev : s->all_events) cudaEventDestroy(ev);
    cudaFree(s->arena_base);
    cudaFree(s->status);
    if (s->scratch) cudaFree(s->scratch);
    delete s;
}

}  // namespace gbfft

using namespace gbfft;

extern "C" {

gbfft_status gbfft_server_create(gbfft_server* out, size_t mem_budget_bytes, int n_streams, int flags) {
    if (!out) return GBFFT_ERR_INVALID_ARG;
    Server* s = nullptr;
    gbfft_status st = server_create(&s, mem_budget_bytes, n_streams, flags);
    *out = reinterpret_cast<gbfft_server>(s);
    return st;
}

gbfft_status gbfft_server_submit(gbfft_server srv, int64_t n, int64_t batch, int direction, const void* host_in,
                                 void* host_out, uint64_t* ticket) {
    if (!srv) return GBFFT_ERR_INVALID_ARG;
    return server_submit(reinterpret_cast<Server*>(srv), n, batch, direction, host_in, host_out, ticket);
}

gbfft_status gbfft_server_prepare(gbfft_server srv, int64_t n, int direction) {
    if (!srv || n < 1) return GBFFT_ERR_INVALID_ARG;
    return server_prepare(reinterpret_cast<Server*>(srv), n, direction);
}

gbfft_status gbfft_server_poll(gbfft_server srv, uint64_t ticket, int* done, double* latency_s) {
    if (!srv) return GBFFT_ERR_INVALID_ARG;
    return server_poll(reinterpret_cast<Server*>(srv), ticket, done, latency_s);
}

gbfft_status gbfft_server_timing(gbfft_server srv, uint64_t ticket, double* queued_s, double* latency_s) {
    if (!srv) return GBFFT_ERR_INVALID_ARG;
    return server_timing(reinterpret_cast<Server*>(srv), ticket, queued_s, latency_s);
}

gbfft_status gbfft_server_wait(gbfft_server srv, uint64_t ticket, double timeout_s) {
    if (!srv || !(timeout_s >= 0)) return GBFFT_ERR_INVALID_ARG;
    return server_wait(reinterpret_cast<Server*>(srv), ticket, timeout_s);
}

gbfft_status gbfft_server_release(gbfft_server srv, uint64_t ticket) {
    if (!srv) return GBFFT_ERR_INVALID_ARG;
    return server_release(reinterpret_cast<Server*>(srv), ticket);
}

gbfft_status gbfft_server_replay(gbfft_server srv, int64_t count, const int64_t* n, const int64_t* batch,
                                 const int* direction, const void* const* host_in, void* const* host_out,
                                 const double* arrival_s, uint64_t* tickets) {
    if (!srv || count < 0 || (count > 0 && (!n || !batch || !direction || !host_in || !host_out || !arrival_s ||
                                            !tickets)))
        return GBFFT_ERR_INVALID_ARG;
    return server_replay(reinterpret_cast<Server*>(srv), count, n, batch, direction, host_in, host_out, arrival_s,
                         tickets);
}

gbfft_status gbfft_server_stats(gbfft_server srv, double* out10) {
    if (!srv || !out10) return GBFFT_ERR_INVALID_ARG;
    server_stats(reinterpret_cast<Server*>(srv), out10, 10);
    return GBFFT_OK;
}

gbfft_status gbfft_server_reset_stats(gbfft_server srv) {
    if (!srv) return GBFFT_ERR_INVALID_ARG;
    server_reset_stats(reinterpret_cast<Server*>(srv));
    return GBFFT_OK;
}

gbfft_status gbfft_server_destroy(gbfft_server srv) {
    if (srv) server_destroy(reinterpret_cast<Server*>(srv));
    return GBFFT_OK;
}

}  // extern "C"
