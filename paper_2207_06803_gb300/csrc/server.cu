// Serving loop: continuous batching of FFT requests under a device-memory budget.
//
// Requests (n, batch, direction, input, output; host or device buffers) are
// submitted from any thread and queued with their arrival time.  One worker
// thread owns the device side:
//   admission   FIFO: the head request is admitted when its slot fits in what
//               is left of a device arena of `budget` bytes (first-fit
//               allocator over one cudaMalloc made at start-up); a request
//               larger than the whole budget is refused at submit time.
//   batching    the requests admitted in one round whose lengths the ragged
//               kernel takes (7-smooth, <= 8192) share, per direction, one
//               slot and ONE persistent ragged launch: their rows are copied
//               in, a queue of (length, rows) items built on the host is
//               uploaded with one copy, the kernel transforms every row in
//               place, the rows are copied back.  Longer lengths are grouped
//               by (n, direction), one slot and one launch each.  Each group
//               goes to the stream with the fewest bytes in flight, so
//               requests that arrive while others are on the GPU are admitted
//               as memory frees up and their copies and kernels overlap.
//   plans       per length the schedule, the ragged length descriptor and the
//               twiddle tables are built once and stay resident.
//   completion  an event recorded after a group's copies back; the worker
//               polls it, stamps the completion time when it finds it
//               complete and frees the slot.  Latency = completion - arrival.
//               With phase timing, events around the copies in, the launch
//               and the copies out split each request's latency into phases
//               on the host clock.  (Host-function callbacks were used first;
//               runs of a few seconds then showed pauses of 40-120 ms in the
//               device-side service of a few hundred requests.)
// Serial mode (one stream, one request per group, one request in flight) is
// the naive queue the batching loop is compared with.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <functional>
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

// Phases of a request's service, in seconds (see gbfft_server_phases).
enum Phase : int {
    kPhQueued = 0,    // admitted - arrival: waiting in the server queue
    kPhHost = 1,      // launched - admitted: the worker issuing the group's copies and launches
    kPhDevWait = 2,   // device start of the group's first copy - launched: waiting behind earlier work
    kPhH2D = 3,       // input copies
    kPhKernel = 4,    // the transform launch(es)
    kPhD2H = 5,       // output copies
    kPhObserve = 6,   // worker seeing the completion - device end of the copies back
    kPhLatency = 7,   // completion seen - arrival
    kNumPhases = 8
};

struct Request {
    uint64_t ticket;
    int64_t n, batch;
    int direction;
    const void* in;
    void* out;
    // Device-visible addresses of in/out (pinned host memory mapped into the device's address space,
    // or device memory): a ragged launch reads and writes them directly, over NVLink-C2C for host
    // memory, without copies.  Null when either buffer is not device-visible.
    const void* din = nullptr;
    void* dout = nullptr;
    Clock::time_point arrival, admitted;
    double latency = 0;
    double queued = 0;  // admitted - arrival: waiting in the server queue
    double phase[kNumPhases] = {};
    bool timed = false;  // phase[] holds device-side phases too
    int state = kQueued;
};

struct Group {
    std::vector<Request*> reqs;
    size_t off = 0, bytes = 0;
    bool ragged = false;       // one ragged launch over requests of several lengths
    bool direct = false;       // the launch reads and writes the requests' own buffers (no slot for rows)
    int direction = GBFFT_FORWARD;
    char* blob = nullptr;      // pinned host copy of the ragged queue (owned while in flight)
    size_t blob_bytes = 0, blob_off = 0;
    int64_t nitems = 0;
    std::vector<size_t> at;    // byte offset of each request's rows in the slot
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;  // recorded after the group's copies back
    cudaEvent_t ph[3] = {};    // with phase timing: before the copies in, after them, after the launch
    Clock::time_point launched, completed;
};

}  // namespace

constexpr size_t kWarmScratchBytes = size_t(4) << 20;  // one row (and its two-pass workspace) up to N = 262144

constexpr size_t kBlobCap = size_t(4) << 20;  // pinned staging for one ragged queue

struct Server {
    int device = 0;
    bool ragged_batching = true;  // requests of lengths <= 8192 share one ragged launch per direction and round
    bool phases = false;          // per-group timing events: device phases of every request
    bool direct_io = true;        // ragged launches on device-visible buffers skip the copies
    RaggedTable* rtable = nullptr;
    std::vector<char*> free_blobs, all_blobs;
    cudaEvent_t ref_ev = nullptr;  // device timeline origin for the phase events
    Clock::time_point ref_host;    // host time of ref_ev
    size_t ragged_groups = 0;
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
    std::vector<cudaEvent_t> free_events, all_events;  // completion and phase events, reused
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
    // Lengths the ragged launches can take get a resident table entry, warmed up the same way.
    if (s->rtable && ragged_supported(n)) {
        int cls = 0;
        const gbfft_status st = ragged_table_add(s->rtable, n, s->tstream, &cls);
        if (st != GBFFT_OK) return st;
        const RaggedSpan span{n, 0, 1};
        std::vector<char> blob(ragged_blob_bytes(8, 1));
        size_t bytes = 0;
        const int64_t nitems = ragged_table_build(s->rtable, &span, 1, blob.data(), blob.size(), &bytes);
        char* d_blob = reinterpret_cast<char*>(s->scratch) + kWarmScratchBytes / 2;
        if (nitems < 0 ||
            cudaMemcpyAsync(d_blob, blob.data(), bytes, cudaMemcpyHostToDevice, s->tstream) != cudaSuccess ||
            ragged_table_launch(s->rtable, dir, s->scratch, d_blob, nitems, s->status, s->tstream) != cudaSuccess)
            return GBFFT_ERR_CUDA;
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

size_t round16(size_t b) { return (b + 15) & ~size_t(15); }

// A request's share of a ragged group's slot: its rows (16-byte aligned).
size_t ragged_share(const Request* r) { return round16(sizeof(float2) * (size_t)r->n * (size_t)r->batch); }

bool can_ragged(const Server* s, const Request* r) {
    return s->rtable && s->ragged_batching && !s->serial && ragged_supported(r->n);
}

// Timing events of a group, recorded only with phase timing on.
void record_phase(Server* s, Group* g, int k) {
    if (s->phases) cudaEventRecord(g->ph[k], g->stream);
}

// Launch a direct ragged group: the queue blob (rows addressed from the first
// request's input, outputs by each item's offset), then one persistent launch
// reading and writing the requests' own buffers.
bool launch_direct_group(Server* s, Group* g) {
    char* base = s->arena_base + g->off;
    bool ok = true;
    record_phase(s, g, 0);
    ok = ok && cudaMemcpyAsync(base + g->blob_off, g->blob, g->blob_bytes, cudaMemcpyHostToDevice, g->stream) ==
                   cudaSuccess;
    record_phase(s, g, 1);
    float2* data = (float2*)const_cast<void*>(g->reqs[0]->din);
    ok = ok && ragged_table_launch(s->rtable, g->direction, data, base + g->blob_off, g->nitems, s->status,
                                   g->stream) == cudaSuccess;
    record_phase(s, g, 2);
    ok = ok && cudaEventRecord(g->ev, g->stream) == cudaSuccess;
    return ok;
}

// Launch a ragged group: copies of every request's rows into the slot, the
// queue blob, one persistent launch over all rows in place, copies back.
bool launch_ragged_group(Server* s, Group* g) {
    char* base = s->arena_base + g->off;
    bool ok = true;
    record_phase(s, g, 0);
    for (size_t i = 0; i < g->reqs.size(); ++i) {
        const Request* r = g->reqs[i];
        ok = ok && cudaMemcpyAsync(base + g->at[i], r->in, sizeof(float2) * (size_t)r->n * (size_t)r->batch,
                                   cudaMemcpyDefault, g->stream) == cudaSuccess;
    }
    ok = ok && cudaMemcpyAsync(base + g->blob_off, g->blob, g->blob_bytes, cudaMemcpyHostToDevice, g->stream) ==
                   cudaSuccess;
    record_phase(s, g, 1);
    ok = ok && ragged_table_launch(s->rtable, g->direction, (float2*)base, base + g->blob_off, g->nitems, s->status,
                                   g->stream) == cudaSuccess;
    record_phase(s, g, 2);
    for (size_t i = 0; i < g->reqs.size(); ++i) {
        const Request* r = g->reqs[i];
        ok = ok && cudaMemcpyAsync(r->out, base + g->at[i], sizeof(float2) * (size_t)r->n * (size_t)r->batch,
                                   cudaMemcpyDefault, g->stream) == cudaSuccess;
    }
    ok = ok && cudaEventRecord(g->ev, g->stream) == cudaSuccess;
    return ok;
}

// Launch one group: H2D of each request into the slot, one transform over
// all rows (in place), D2H of each request, completion stamp.
// A request a per-length group can transform where its buffers are: both
// device-visible and 16-byte aligned (the row kernels move 16-byte units).
bool direct_single(const Server* s, const Request* r) {
    return s->direct_io && !s->serial && r->din && ((uintptr_t)r->din & 15u) == 0 && ((uintptr_t)r->dout & 15u) == 0;
}

// Arena bytes a request's group needs: its rows (staged) or only the two-pass
// workspace (direct).
size_t group_bytes(const Server* s, int64_t n, int64_t rows, bool two_pass, bool direct) {
    (void)s;
    if (!direct) return slot_bytes(n, rows, two_pass);
    return two_pass ? ((sizeof(float2) * (size_t)n * (size_t)rows + 255) & ~size_t(255)) : 256;
}

bool launch_group(Server* s, Group* g, ServerPlan* sp, int64_t n, int dir, int64_t rows) {
    float2* data = (float2*)(s->arena_base + g->off);
    const size_t row_bytes = sizeof(float2) * (size_t)n;
    bool ok = true;
    size_t at = 0;
    record_phase(s, g, 0);
    if (g->direct) {  // each request transformed where it is; the slot holds the two-pass workspace only
        record_phase(s, g, 1);
        for (Request* r : g->reqs) {
            const float2* din = (const float2*)r->din;
            float2* dout = (float2*)r->dout;
            if (!sp->two_pass) {
                ok = ok && launch_rows(*sp->rv, dir, din, dout, sp->tw, (long long)r->batch, sp->grid_cap, g->stream,
                                       s->status) == cudaSuccess;
            } else {
                ok = ok && launch_cols(*sp->cm, 1, dir, din, data, sp->tw_m, sp->post, (long long)r->batch,
                                       (int)sp->k, g->stream) == cudaSuccess;
                ok = ok && launch_cols(*sp->ck, 2, dir, data, dout, sp->tw_k, nullptr, (long long)r->batch,
                                       (int)sp->m, g->stream) == cudaSuccess;
            }
        }
        record_phase(s, g, 2);
        return ok && cudaEventRecord(g->ev, g->stream) == cudaSuccess;
    }
    for (Request* r : g->reqs) {
        ok = ok && cudaMemcpyAsync((char*)data + at, r->in, row_bytes * (size_t)r->batch, cudaMemcpyDefault,
                                   g->stream) == cudaSuccess;
        at += row_bytes * (size_t)r->batch;
    }
    record_phase(s, g, 1);
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
    record_phase(s, g, 2);
    at = 0;
    for (Request* r : g->reqs) {
        ok = ok && cudaMemcpyAsync(r->out, (char*)data + at, row_bytes * (size_t)r->batch, cudaMemcpyDefault,
                                   g->stream) == cudaSuccess;
        at += row_bytes * (size_t)r->batch;
    }
    ok = ok && cudaEventRecord(g->ev, g->stream) == cudaSuccess;
    return ok;
}

cudaEvent_t acquire_event(Server* s) {
    if (s->free_events.empty()) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, s->phases ? cudaEventDefault : cudaEventDisableTiming) != cudaSuccess)
            return nullptr;
        s->all_events.push_back(ev);
        return ev;
    }
    cudaEvent_t ev = s->free_events.back();
    s->free_events.pop_back();
    return ev;
}

char* acquire_blob(Server* s) {
    if (s->free_blobs.empty()) {
        char* b = nullptr;
        if (cudaHostAlloc(&b, kBlobCap, cudaHostAllocDefault) != cudaSuccess) return nullptr;
        s->all_blobs.push_back(b);
        return b;
    }
    char* b = s->free_blobs.back();
    s->free_blobs.pop_back();
    return b;
}

// Host time of a device event (ref_ev's host time plus the device interval).
double event_seconds_after(Server* s, cudaEvent_t ev, Clock::time_point t0) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->ref_ev, ev) != cudaSuccess) return 0.0;
    return seconds_since(t0, s->ref_host) + 1e-3 * (double)ms;
}

void release_group_resources(Server* s, Group* g) {
    s->free_events.push_back(g->ev);
    for (cudaEvent_t e : g->ph)
        if (e) s->free_events.push_back(e);
    if (g->blob) s->free_blobs.push_back(g->blob);
    g->blob = nullptr;
    s->arena->release(g->off, g->bytes);
}

void retire(Server* s, Group* g) {
    g->completed = Clock::now();
    for (Request* r : g->reqs) {
        r->latency = seconds_since(r->arrival, g->completed);
        r->queued = seconds_since(r->arrival, r->admitted);
        double* ph = r->phase;
        ph[kPhQueued] = r->queued;
        ph[kPhHost] = seconds_since(r->admitted, g->launched);
        ph[kPhLatency] = r->latency;
        if (s->phases) {
            const double t0 = event_seconds_after(s, g->ph[0], r->arrival);
            const double t1 = event_seconds_after(s, g->ph[1], r->arrival);
            const double t2 = event_seconds_after(s, g->ph[2], r->arrival);
            const double t3 = event_seconds_after(s, g->ev, r->arrival);
            ph[kPhDevWait] = t0 - seconds_since(r->arrival, g->launched);
            ph[kPhH2D] = t1 - t0;
            ph[kPhKernel] = t2 - t1;
            ph[kPhD2H] = t3 - t2;
            ph[kPhObserve] = r->latency - t3;
            r->timed = true;
        }
        r->state = kDone;
        s->latencies.push_back(r->latency);
        s->bytes_done += 16.0 * (double)r->n * (double)r->batch;
    }
    s->win_last = g->completed;
    release_group_resources(s, g);
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
                retire(s, g);
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
        std::map<std::pair<int64_t, int>, std::vector<Request*>> groups;  // per (n, direction)
        std::map<std::pair<int, int>, std::vector<Request*>> rgroups;      // ragged, per (direction, direct)
        size_t pending_bytes = 0;
        while (!s->queue.empty()) {
            if (s->serial && (inflight_reqs + admitted.size()) >= 1) break;
            Request* r = s->queue.front();
            const bool rg = can_ragged(s, r);
            const bool direct = rg && s->direct_io && r->din;
            const size_t need = rg ? (direct ? 0 : ragged_share(r)) + 40 * (size_t)r->batch + 512
                                   : group_bytes(s, r->n, r->batch, needs_two_pass(r->n), direct_single(s, r)) + 256;
            if (s->arena->used() + pending_bytes + need > s->arena->size()) break;
            s->queue.pop_front();
            admitted.push_back(r);
            pending_bytes += need;
            if (rg) rgroups[{r->direction, (s->direct_io && r->din) ? 1 : 0}].push_back(r);
            else groups[{r->n, r->direction}].push_back(r);
        }
        // 3. one slot and one launch per ragged direction group and per (n, direction) group; a group
        //    whose slot does not fit contiguously (fragmentation) is retried request by request, and
        //    what still does not fit returns to the queue front.
        std::vector<Request*> retry;
        auto fail_reqs = [&](const std::vector<Request*>& reqs, gbfft_status st) {
            s->error = st;
            for (Request* r : reqs) r->state = kFailed;
            s->cv.notify_all();
        };
        // Start a prepared group (slot size in g->bytes): slot, events, stream, then the launch
        // without the lock.  false: no slot (the caller retries smaller).
        auto start = [&](std::unique_ptr<Group> g, const std::function<bool(Group*)>& launch) -> bool {
            if (!s->arena->alloc(g->bytes, &g->off)) {
                if (g->blob) s->free_blobs.push_back(g->blob);
                return false;
            }
            g->ev = acquire_event(s);
            bool ev_ok = g->ev != nullptr;
            if (s->phases)
                for (cudaEvent_t& e : g->ph) ev_ok = ev_ok && (e = acquire_event(s)) != nullptr;
            if (!ev_ok) {
                for (cudaEvent_t e : g->ph)
                    if (e) s->free_events.push_back(e);
                if (g->ev) s->free_events.push_back(g->ev);
                if (g->blob) s->free_blobs.push_back(g->blob);
                s->arena->release(g->off, g->bytes);
                fail_reqs(g->reqs, GBFFT_ERR_CUDA);
                return true;
            }
            // The stream with the fewest bytes in flight: a small group does not queue behind a large one
            // when another stream is idle (ties go round robin).
            {
                std::vector<size_t> load(s->streams.size(), 0);
                for (auto& f : s->inflight)
                    for (size_t k = 0; k < s->streams.size(); ++k)
                        if (f->stream == s->streams[k]) load[k] += f->bytes;
                size_t best = (size_t)s->next_stream;
                for (size_t j = 0; j < s->streams.size(); ++j) {
                    const size_t k = ((size_t)s->next_stream + j) % s->streams.size();
                    if (load[k] < load[best]) best = k;
                }
                g->stream = s->streams[best];
                s->next_stream = (int)((best + 1) % s->streams.size());
            }
            const Clock::time_point now = Clock::now();
            for (Request* r : g->reqs) {
                r->state = kRunning;
                r->admitted = now;
            }
            // The copies and launches run without the lock: the group's requests are Running (no other
            // thread changes or releases them), its slot and events are the worker's, and submissions
            // need not wait behind a group's API calls.
            lk.unlock();
            const bool launched = launch(g.get());
            g->launched = Clock::now();
            lk.lock();
            if (!launched) {
                cudaStreamSynchronize(g->stream);
                release_group_resources(s, g.get());
                fail_reqs(g->reqs, GBFFT_ERR_CUDA);
                return true;
            }
            ++s->groups_launched;
            if (g->ragged) ++s->ragged_groups;
            s->inflight.push_back(std::move(g));
            return true;
        };
        auto start_group = [&](std::vector<Request*> reqs, int64_t n, int dir, ServerPlan* sp) -> bool {
            int64_t rows = 0;
            for (Request* r : reqs) rows += r->batch;
            auto g = std::make_unique<Group>();
            g->reqs = std::move(reqs);
            g->direction = dir;
            g->direct = true;
            for (Request* r : g->reqs) g->direct = g->direct && direct_single(s, r);
            g->bytes = group_bytes(s, n, rows, sp->two_pass, g->direct);
            return start(std::move(g), [&](Group* gg) { return launch_group(s, gg, sp, n, dir, rows); });
        };
        auto start_ragged = [&](std::vector<Request*> reqs, int dir, bool direct) -> int {  // 1 started, 0 no slot,
                                                                                             // -1 no queue
            auto g = std::make_unique<Group>();
            g->ragged = true;
            g->direct = direct;
            g->direction = dir;
            g->reqs = std::move(reqs);
            std::vector<RaggedSpan> spans;
            size_t data = 0;
            if (direct) {  // element offsets from the first request's input; outputs by their distance
                const char* base = (const char*)g->reqs[0]->din;
                for (Request* r : g->reqs)
                    spans.push_back(RaggedSpan{r->n, (long long)(((const char*)r->din - base) / (long long)sizeof(float2)),
                                               r->batch,
                                               (long long)(((char*)r->dout - (const char*)r->din) / (long long)sizeof(float2))});
            } else {
                for (Request* r : g->reqs) {
                    g->at.push_back(data);
                    spans.push_back(RaggedSpan{r->n, (long long)(data / sizeof(float2)), r->batch, 0});
                    data += ragged_share(r);
                }
            }
            g->blob = acquire_blob(s);
            if (!g->blob) return -1;
            g->nitems = ragged_table_build(s->rtable, spans.data(), (int64_t)spans.size(), g->blob, kBlobCap,
                                           &g->blob_bytes);
            if (g->nitems < 0) {
                s->free_blobs.push_back(g->blob);
                return -1;
            }
            g->blob_off = (data + 255) & ~size_t(255);
            g->bytes = g->blob_off + g->blob_bytes;
            return start(std::move(g), [&](Group* gg) {
                       return gg->direct ? launch_direct_group(s, gg) : launch_ragged_group(s, gg);
                   }) ? 1 : 0;
        };
        auto start_per_length = [&](const std::vector<Request*>& reqs) {
            std::map<std::pair<int64_t, int>, std::vector<Request*>> by;
            for (Request* r : reqs) by[{r->n, r->direction}].push_back(r);
            for (auto& kv : by) {
                ServerPlan* sp = nullptr;
                const gbfft_status st = get_plan(s, kv.first.first, kv.first.second, &sp);
                if (st != GBFFT_OK) {
                    fail_reqs(kv.second, st);
                    continue;
                }
                if (start_group(kv.second, kv.first.first, kv.first.second, sp)) continue;
                for (Request* r : kv.second)
                    if (!start_group({r}, kv.first.first, kv.first.second, sp)) retry.push_back(r);
            }
        };
        for (auto& kv : rgroups) {
            std::vector<Request*> ok_reqs;
            for (Request* r : kv.second) {  // every length needs its table entry (built once, then resident)
                ServerPlan* sp = nullptr;
                const gbfft_status st = get_plan(s, r->n, r->direction, &sp);
                if (st != GBFFT_OK) fail_reqs({r}, st);
                else ok_reqs.push_back(r);
            }
            if (ok_reqs.empty()) continue;
            const int dir = kv.first.first;
            const bool direct = kv.first.second != 0;
            const int res = start_ragged(ok_reqs, dir, direct);
            if (res == 1) continue;
            if (res == 0) {  // no contiguous slot: halves, then single requests
                std::vector<Request*> a(ok_reqs.begin(), ok_reqs.begin() + (std::ptrdiff_t)(ok_reqs.size() / 2));
                std::vector<Request*> b(ok_reqs.begin() + (std::ptrdiff_t)(ok_reqs.size() / 2), ok_reqs.end());
                for (auto* half : {&a, &b}) {
                    if (half->empty() || start_ragged(*half, dir, direct) == 1) continue;
                    for (Request* r : *half)
                        if (start_ragged({r}, dir, direct) != 1) retry.push_back(r);
                }
                continue;
            }
            start_per_length(ok_reqs);  // the queue did not fit the staging blob
        }
        for (auto& kv : groups) start_per_length(kv.second);
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
    s->serial = (flags & GBFFT_SERVER_SERIAL) != 0;
    s->phases = (flags & GBFFT_SERVER_PHASES) != 0;
    s->ragged_batching = (flags & GBFFT_SERVER_PER_LENGTH) == 0;
    s->direct_io = (flags & GBFFT_SERVER_STAGED) == 0;
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
    if (s->ragged_batching && !s->serial && ragged_table_create(&s->rtable) != GBFFT_OK) {
        for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
        cudaFree(s->arena_base);
        delete s;
        return GBFFT_ERR_OOM;
    }
    if (s->phases) {  // the origin of the device timeline, placed on the host clock
        if (cudaEventCreate(&s->ref_ev) != cudaSuccess || cudaEventRecord(s->ref_ev, s->tstream) != cudaSuccess ||
            cudaEventSynchronize(s->ref_ev) != cudaSuccess) {
            ragged_table_destroy(s->rtable);
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            cudaFree(s->arena_base);
            delete s;
            return GBFFT_ERR_CUDA;
        }
        s->ref_host = Clock::now();
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return GBFFT_OK;
}

// The address at which the device reaches `p` (device or managed memory, or
// page-locked host memory mapped into the device's address space), or null.
const void* device_visible(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged || a.type == cudaMemoryTypeHost)
        return a.devicePointer;
    return nullptr;
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
    {
        const void* di = device_visible(in);
        void* dd = const_cast<void*>(device_visible(out));
        if (di && dd && ((uintptr_t)di & 7u) == 0 && ((uintptr_t)dd & 7u) == 0) {
            r->din = di;
            r->dout = dd;
        }
    }
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

gbfft_status server_phases(Server* s, uint64_t ticket, double* out) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return GBFFT_ERR_NOT_FOUND;
    const Request* r = it->second.get();
    if (r->state != kDone) return GBFFT_ERR_INVALID_ARG;
    for (int k = 0; k < kNumPhases; ++k) out[k] = r->phase[k];
    if (!r->timed)
        for (int k : {kPhDevWait, kPhH2D, kPhKernel, kPhD2H, kPhObserve}) out[k] = std::nan("");
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
    if (s->ref_ev) cudaEventDestroy(s->ref_ev);
    for (char* b : s->all_blobs) cudaFreeHost(b);
    ragged_table_destroy(s->rtable);
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

gbfft_status gbfft_server_submit(gbfft_server srv, int64_t n, int64_t batch, int direction, const void* host_or_dev_in,
                                 void* host_or_dev_out, uint64_t* ticket) {
    if (!srv) return GBFFT_ERR_INVALID_ARG;
    return server_submit(reinterpret_cast<Server*>(srv), n, batch, direction, host_or_dev_in, host_or_dev_out,
                         ticket);
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

gbfft_status gbfft_server_phases(gbfft_server srv, uint64_t ticket, double* out8) {
    if (!srv || !out8) return GBFFT_ERR_INVALID_ARG;
    return server_phases(reinterpret_cast<Server*>(srv), ticket, out8);
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
