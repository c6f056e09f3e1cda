// Ragged-batch plans: the persistent kernel of ragged.cuh, its work queue,
// the CUDA graph that launches it, and the tile-shape autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "internal.h"
#include "ragged.cuh"

namespace gbfft {

namespace {

struct ClassInfo {
    int n, t, ps, nstages;
    int radix[kMaxStages];
};

template <int... Rs>
constexpr int count_of() {
    return (int)sizeof...(Rs);
}

#define GBFFT_RAGGED_INFO(idx, N, T, PS, ...) ClassInfo{N, T, PS, count_of<__VA_ARGS__>(), {__VA_ARGS__}},
const ClassInfo kClasses[kRaggedCases] = {GBFFT_RAGGED_CLASSES(GBFFT_RAGGED_INFO)};
#undef GBFFT_RAGGED_INFO

int class_of(int64_t n) {
    for (int c = 0; c < kRaggedCases; ++c)
        if (kClasses[c].n == n) return c;
    return -1;
}

int class_smem_bytes(int c) {
    const ClassInfo& k = kClasses[c];
    const int elems = k.t * k.n;
    return (int)sizeof(float2) * ((elems - 1) + ((elems - 1) >> k.ps) + 1);
}

}  // namespace

struct RaggedState {
    int64_t count = 0;
    int64_t total = 0;  // elements spanned by the transforms (max offset + n)
    std::vector<int64_t> n, off;
    std::vector<std::vector<int64_t>> members;  // transform indices per class
    int split[kRaggedCases];                  // tile shape: rows per item = T_c / split[c]
    int order = 1;                              // queue order: 0 = heaviest item first, 1 = grouped by class
    std::vector<RaggedItem> items;
    std::vector<long long> row_offs;
    RaggedItem* d_items = nullptr;
    long long* d_offs = nullptr;
    float2* d_tw = nullptr;
    int* d_twoff = nullptr;
    int* d_counter = nullptr;
    int smem = 0;
    int grid = 0;
    long long wait_ns = 200000000LL;  // 200 ms bound on any ready-wait
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t knode = nullptr;
    const void* g_in = nullptr;
    void* g_out = nullptr;
};

static void ragged_release_graph(RaggedState* r) {
    if (r->exec) cudaGraphExecDestroy(r->exec);
    if (r->graph) cudaGraphDestroy(r->graph);
    r->exec = nullptr;
    r->graph = nullptr;
    r->knode = nullptr;
}

void ragged_destroy(RaggedState* r) {
    if (!r) return;
    ragged_release_graph(r);
    if (r->d_items) cudaFree(r->d_items);
    if (r->d_offs) cudaFree(r->d_offs);
    if (r->d_tw) cudaFree(r->d_tw);
    if (r->d_twoff) cudaFree(r->d_twoff);
    if (r->d_counter) cudaFree(r->d_counter);
    delete r;
}

// Items from the current tile shapes: class groups cut into items of
// ceil(T_c / split_c) rows.  Order 0: all items by work (rows * N log N),
// heaviest first (longest-processing-time list scheduling).  Order 1: items
// stay grouped by class, classes ordered by item work, heaviest first, so
// that CTAs claiming neighbouring items run the same class's code (the
// kernel holds one fully unrolled schedule per class; interleaving classes
// thrashes the instruction cache).
static gbfft_status ragged_build_items(RaggedState* r) {
    r->items.clear();
    r->row_offs.clear();
    struct Pending {
        double cost;
        int cls;
        std::vector<long long> rows;
    };
    std::vector<Pending> pend;
    for (int c = 0; c < kRaggedCases; ++c) {
        const std::vector<int64_t>& mem = r->members[c];
        if (mem.empty()) continue;
        int rows = kClasses[c].t / r->split[c];
        if (rows < 1) rows = 1;
        for (size_t i = 0; i < mem.size(); i += rows) {
            Pending p;
            p.cls = c;
            const size_t e = std::min(mem.size(), i + (size_t)rows);
            for (size_t k = i; k < e; ++k) p.rows.push_back((long long)r->off[mem[k]]);
            p.cost = (double)p.rows.size() * kClasses[c].n * std::log2((double)kClasses[c].n);
            pend.push_back(std::move(p));
        }
    }
    if (r->order == 0) {
        std::stable_sort(pend.begin(), pend.end(), [](const Pending& a, const Pending& b) { return a.cost > b.cost; });
    } else {
        std::vector<double> cls_cost(kRaggedCases, 0.0);
        for (const Pending& p : pend) cls_cost[p.cls] = std::max(cls_cost[p.cls], p.cost);
        std::stable_sort(pend.begin(), pend.end(), [&](const Pending& a, const Pending& b) {
            if (a.cls != b.cls) return cls_cost[a.cls] > cls_cost[b.cls] || (cls_cost[a.cls] == cls_cost[b.cls] && a.cls > b.cls);
            return a.cost > b.cost;
        });
    }
    for (const Pending& p : pend) {
        RaggedItem it;
        it.cls = p.cls;
        it.count = (int)p.rows.size();
        it.first = (int)r->row_offs.size();
        it.ready = 1;
        r->items.push_back(it);
        r->row_offs.insert(r->row_offs.end(), p.rows.begin(), p.rows.end());
    }
    if (r->d_items) cudaFree(r->d_items);
    if (r->d_offs) cudaFree(r->d_offs);
    r->d_items = nullptr;
    r->d_offs = nullptr;
    if (cudaMalloc(&r->d_items, sizeof(RaggedItem) * r->items.size()) != cudaSuccess ||
        cudaMalloc(&r->d_offs, sizeof(long long) * r->row_offs.size()) != cudaSuccess) {
        cudaGetLastError();
        return GBFFT_ERR_OOM;
    }
    if (cudaMemcpy(r->d_items, r->items.data(), sizeof(RaggedItem) * r->items.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(r->d_offs, r->row_offs.data(), sizeof(long long) * r->row_offs.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return GBFFT_ERR_CUDA;
    return GBFFT_OK;
}

static cudaError_t ragged_launch(RaggedState* r, int direction, const void* in, void* out, int* status,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(r->d_counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    int nitems = (int)r->items.size();
    const float2* pin = (const float2*)in;
    float2* pout = (float2*)out;
    void* args[] = {(void*)&pin, (void*)&pout, (void*)&r->d_items, (void*)&nitems, (void*)&r->d_offs,
                    (void*)&r->d_tw,  (void*)&r->d_twoff, (void*)&r->d_counter, (void*)&status, (void*)&r->wait_ns};
    const void* fn = direction == GBFFT_FORWARD ? ragged_kernel_fwd() : ragged_kernel_inv();
    int grid = std::min<int>(r->grid, nitems > 0 ? nitems : 1);
    return cudaLaunchKernel(fn, dim3(grid), dim3(kRaggedThreads), args, (size_t)r->smem, s);
}

gbfft_status ragged_create(RaggedState** out, const int64_t* n, const int64_t* offsets, int64_t count) {
    *out = nullptr;
    if (!n || !offsets || count < 1 || count > (int64_t)1 << 30) return GBFFT_ERR_INVALID_ARG;
    RaggedState* r = new (std::nothrow) RaggedState();
    if (!r) return GBFFT_ERR_OOM;
    r->count = count;
    r->n.assign(n, n + count);
    r->off.assign(offsets, offsets + count);
    r->members.assign(kRaggedCases, {});
    for (int c = 0; c < kRaggedCases; ++c) r->split[c] = 1;
    std::vector<std::pair<int64_t, int64_t>> spans;
    spans.reserve(count);
    for (int64_t i = 0; i < count; ++i) {
        if (n[i] < 1 || offsets[i] < 0) {
            delete r;
            return GBFFT_ERR_INVALID_ARG;
        }
        const int c = class_of(n[i]);
        if (c < 0) {
            delete r;
            return GBFFT_ERR_UNSUPPORTED_SIZE;
        }
        r->members[c].push_back(i);
        spans.push_back({offsets[i], offsets[i] + n[i]});
        r->total = std::max(r->total, offsets[i] + n[i]);
    }
    std::sort(spans.begin(), spans.end());
    for (size_t i = 1; i < spans.size(); ++i) {
        if (spans[i].first < spans[i - 1].second) {
            delete r;
            return GBFFT_ERR_OVERLAP;
        }
    }
    // Stage-twiddle blocks of every compiled case whose length is present
    // (default and alternative schedules), concatenated.
    std::vector<char> present(kRaggedCases, 0);
    for (int c = 0; c < kRaggedCases; ++c)
        for (int d = 0; d < kRaggedCases; ++d)
            if (!r->members[d].empty() && kClasses[d].n == kClasses[c].n) present[c] = 1;
    std::vector<int> twoff(kRaggedCases, 0);
    int tw_total = 0;
    r->smem = 0;
    for (int c = 0; c < kRaggedCases; ++c) {
        if (!present[c]) continue;
        twoff[c] = tw_total;
        tw_total += stage_twiddle_count(kClasses[c].radix, kClasses[c].nstages);
        r->smem = std::max(r->smem, class_smem_bytes(c));
    }
    gbfft_status st = GBFFT_OK;
    if (cudaMalloc(&r->d_tw, sizeof(float2) * (size_t)std::max(tw_total, 1)) != cudaSuccess ||
        cudaMalloc(&r->d_twoff, sizeof(int) * kRaggedCases) != cudaSuccess ||
        cudaMalloc(&r->d_counter, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        st = GBFFT_ERR_OOM;
    }
    for (int c = 0; st == GBFFT_OK && c < kRaggedCases; ++c) {
        if (!present[c]) continue;
        if (launch_stage_twiddles(r->d_tw + twoff[c], kClasses[c].n, kClasses[c].radix, kClasses[c].nstages, 0) !=
            cudaSuccess)
            st = GBFFT_ERR_CUDA;
    }
    if (st == GBFFT_OK &&
        cudaMemcpy(r->d_twoff, twoff.data(), sizeof(int) * kRaggedCases, cudaMemcpyHostToDevice) != cudaSuccess)
        st = GBFFT_ERR_CUDA;
    if (st == GBFFT_OK) {
        const void* ks[2] = {ragged_kernel_fwd(), ragged_kernel_inv()};
        int dev = 0, sms = 0, per_sm = 0;
        for (const void* k : ks)
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, r->smem) != cudaSuccess)
                st = GBFFT_ERR_CUDA;
        if (st == GBFFT_OK &&
            (cudaGetDevice(&dev) != cudaSuccess ||
             cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
             cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks[0], kRaggedThreads, (size_t)r->smem) !=
                 cudaSuccess ||
             per_sm < 1))
            st = GBFFT_ERR_CUDA;
        r->grid = per_sm * sms;
    }
    if (st == GBFFT_OK) st = ragged_build_items(r);
    if (st == GBFFT_OK && cudaDeviceSynchronize() != cudaSuccess) st = GBFFT_ERR_CUDA;
    if (st != GBFFT_OK) {
        ragged_destroy(r);
        return st;
    }
    *out = r;
    return GBFFT_OK;
}

int64_t ragged_total(const RaggedState* r) { return r->total; }

// Capture (once per set of buffers) the counter reset + persistent launch into
// a CUDA graph; later calls with other buffers patch the kernel node's
// parameters in the instantiated graph.
gbfft_status ragged_execute(RaggedState* r, int direction, const void* in, void* out, int* status, cudaStream_t s) {
    if (!r->exec) {
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return GBFFT_ERR_CUDA;
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        cudaError_t le = ok ? ragged_launch(r, direction, in, out, status, cs) : cudaErrorUnknown;
        cudaGraph_t g = nullptr;
        const bool ended = cudaStreamEndCapture(cs, &g) == cudaSuccess;
        cudaStreamDestroy(cs);
        if (!ok || le != cudaSuccess || !ended || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return GBFFT_ERR_CUDA;
        }
        r->graph = g;
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(g, nodes.data(), &nn);
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) r->knode = nd;
        }
        if (!r->knode || cudaGraphInstantiate(&r->exec, g, 0) != cudaSuccess) {
            ragged_release_graph(r);
            cudaGetLastError();
            return GBFFT_ERR_CUDA;
        }
        r->g_in = in;
        r->g_out = out;
    } else if (in != r->g_in || out != r->g_out) {
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(r->knode, &kp) != cudaSuccess) return GBFFT_ERR_CUDA;
        const float2* pin = (const float2*)in;
        float2* pout = (float2*)out;
        void** a = kp.kernelParams;
        // kernelParams points at copies owned by the graph node; build fresh ones.
        int nitems = (int)r->items.size();
        void* args[] = {(void*)&pin, (void*)&pout, (void*)&r->d_items, (void*)&nitems, (void*)&r->d_offs,
                        (void*)&r->d_tw,  (void*)&r->d_twoff, (void*)&r->d_counter, (void*)&status,
                        (void*)&r->wait_ns};
        (void)a;
        kp.kernelParams = args;
        if (cudaGraphExecKernelNodeSetParams(r->exec, r->knode, &kp) != cudaSuccess ||
            cudaGraphKernelNodeSetParams(r->knode, &kp) != cudaSuccess)
            return GBFFT_ERR_CUDA;
        r->g_in = in;
        r->g_out = out;
    }
    return cudaGraphLaunch(r->exec, s) == cudaSuccess ? GBFFT_OK : GBFFT_ERR_CUDA;
}

// Direct (uncaptured) launch, used by the autotuner and available for comparison.
gbfft_status ragged_execute_direct(RaggedState* r, int direction, const void* in, void* out, int* status,
                                   cudaStream_t s) {
    return ragged_launch(r, direction, in, out, status, s) == cudaSuccess ? GBFFT_OK : GBFFT_ERR_CUDA;
}

int64_t ragged_num_items(const RaggedState* r) { return (int64_t)r->items.size(); }

gbfft_status ragged_set_item_ready(RaggedState* r, int64_t item, int ready) {
    if (item < 0 || item >= (int64_t)r->items.size()) return GBFFT_ERR_NOT_FOUND;
    r->items[item].ready = ready;
    return cudaMemcpy(&r->d_items[item].ready, &ready, sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess
               ? GBFFT_OK
               : GBFFT_ERR_CUDA;
}

void ragged_set_wait_ns(RaggedState* r, long long ns) {
    r->wait_ns = ns;
    ragged_release_graph(r);  // the limit is a kernel argument baked into the graph
}

// Autotuner: queue order, then coordinate descent over the rows-per-item
// split of each class (1, 2, 4, 8), heaviest classes first, then each
// length's compiled alternative radix schedules, timing the whole direct
// launch with CUDA events (median of `reps`).  Keeps the best choices and
// rebuilds the queue; the graph is re-captured on the next execute.
gbfft_status ragged_autotune(RaggedState* r, int direction, const void* in, void* out, int* status, int reps,
                             float* best_ms) {
    cudaStream_t s;
    cudaEvent_t e0, e1;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return GBFFT_ERR_CUDA;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto measure = [&](float* ms) -> gbfft_status {
        gbfft_status st = ragged_build_items(r);
        if (st != GBFFT_OK) return st;
        std::vector<float> t;
        for (int i = 0; i < reps + 1; ++i) {
            cudaEventRecord(e0, s);
            if (ragged_launch(r, direction, in, out, status, s) != cudaSuccess) return GBFFT_ERR_CUDA;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return GBFFT_ERR_CUDA;
            float v = 0.f;
            cudaEventElapsedTime(&v, e0, e1);
            if (i > 0) t.push_back(v);  // first run warms up
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return GBFFT_OK;
    };
    if (reps < 1) reps = 1;
    float best = 0.f;
    gbfft_status st = measure(&best);
    {
        const int keep = r->order;
        r->order = 1 - keep;
        float ms = 0.f;
        if (st == GBFFT_OK) st = measure(&ms);
        if (st == GBFFT_OK && ms < best) best = ms;
        else r->order = keep;
    }
    std::vector<int> order;
    for (int c = 0; c < kRaggedCases; ++c)
        if (!r->members[c].empty()) order.push_back(c);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return (double)r->members[a].size() * kClasses[a].n > (double)r->members[b].size() * kClasses[b].n;
    });
    for (int c : order) {
        if (st != GBFFT_OK) break;
        const int keep = r->split[c];
        int best_split = keep;
        for (int sp : {1, 2, 4, 8}) {
            if (sp == keep || kClasses[c].t / sp < 1) continue;
            r->split[c] = sp;
            float ms = 0.f;
            st = measure(&ms);
            if (st != GBFFT_OK) break;
            if (ms < best) {
                best = ms;
                best_split = sp;
            }
        }
        r->split[c] = best_split;
    }
    // Radix schedule per length: move a length's transforms to each compiled
    // alternative case and keep the fastest.
    std::vector<int64_t> tuned;
    for (int c = 0; st == GBFFT_OK && c < kRaggedCases; ++c) {
        if (r->members[c].empty()) continue;
        if (std::find(tuned.begin(), tuned.end(), kClasses[c].n) != tuned.end()) continue;
        tuned.push_back(kClasses[c].n);
        int cur = c;
        for (int a = 0; a < kRaggedCases && st == GBFFT_OK; ++a) {
            if (a == cur || kClasses[a].n != kClasses[c].n || !r->members[a].empty()) continue;
            r->members[a].swap(r->members[cur]);
            if (kClasses[a].t == kClasses[cur].t) r->split[a] = r->split[cur];  // same tile shape
            float ms = 0.f;
            st = measure(&ms);
            if (st == GBFFT_OK && ms < best) {
                best = ms;
                cur = a;
            } else {
                r->members[cur].swap(r->members[a]);
            }
        }
    }
    if (st == GBFFT_OK) st = ragged_build_items(r);
    ragged_release_graph(r);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (best_ms) *best_ms = best;
    return st;
}

int ragged_queue_order(const RaggedState* r) { return r->order; }

// The case currently used for length n (the one holding its transforms).
static int case_in_use(const RaggedState* r, int64_t n) {
    for (int c = 0; c < kRaggedCases; ++c)
        if (kClasses[c].n == n && !r->members[c].empty()) return c;
    return -1;
}

int ragged_class_split(const RaggedState* r, int64_t n) {
    const int c = case_in_use(r, n);
    return c < 0 ? 0 : r->split[c];
}

int ragged_schedule(const RaggedState* r, int64_t n, int* radix) {
    const int c = case_in_use(r, n);
    if (c < 0) return 0;
    for (int i = 0; i < kClasses[c].nstages; ++i) radix[i] = kClasses[c].radix[i];
    return kClasses[c].nstages;
}

bool ragged_supported(int64_t n) { return class_of(n) >= 0; }

}  // namespace gbfft
