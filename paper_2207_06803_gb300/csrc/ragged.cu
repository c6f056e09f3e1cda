// Ragged-batch plans: the persistent kernel of ragged.cuh, its work queue and
// per-length schedules, the CUDA graph that launches it, and the autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <iterator>
#include <map>
#include <new>
#include <vector>

#include "internal.h"
#include "ragged.cuh"

namespace gbfft {

namespace {

// Candidate radix schedules of a length n = 2^a 3^b 5^c 7^d <= 8192, the
// default first: odd radices first, then the power-of-two part as radix-16
// stages with the remainder first or last, or as radix-8 stages; powers of two
// up to 16 use two stages so that both HBM passes are coalesced.  Empty if n
// has another prime factor.
std::vector<std::vector<int>> schedules_of(int64_t n) {
    std::vector<std::vector<int>> out;
    if (n < 1 || n > kRaggedMaxN) return out;
    std::vector<int> odd;
    int64_t m = n;
    for (int p : {3, 5, 7})
        while (m % p == 0) {
            odd.push_back(p);
            m /= p;
        }
    int a = 0;
    while (m % 2 == 0) {
        ++a;
        m /= 2;
    }
    if (m != 1) return out;
    auto add = [&](std::vector<int> pw, bool front) {
        std::vector<int> sch = odd;
        sch.insert(sch.end(), pw.begin(), pw.end());
        if ((int)sch.size() > kRaggedMaxStages) return;
        for (const auto& c : out)
            if (c == sch) return;
        if (front) out.insert(out.begin(), sch);
        else out.push_back(sch);
    };
    auto pieces = [](int a, int unit, bool rem_first) {
        std::vector<int> v;
        const int full = a / unit, rem = a % unit;
        if (rem && rem_first) v.push_back(1 << rem);
        for (int i = 0; i < full; ++i) v.push_back(1 << unit);
        if (rem && !rem_first) v.push_back(1 << rem);
        return v;
    };
    add(pieces(a, 4, true), false);
    add(pieces(a, 4, false), false);
    add(pieces(a, 3, false), false);
    add(pieces(a, 3, true), false);
    if (odd.empty() && a == 3) add({2, 4}, true);
    if (odd.empty() && a == 4) add({4, 4}, true);
    return out;
}

}  // namespace

struct RaggedLenState {
    int64_t n = 0;
    std::vector<int64_t> members;               // transform indices of this length
    std::vector<std::vector<int>> cands;        // candidate schedules
    int runtime_cands = 0;                      // the first runtime_cands run on the run-time engine
    std::vector<int> tw_base;                   // twiddle-table offset of each candidate
    int cand = 0;                               // schedule in use by the run-time engine
    int split = 1;                              // tile shape: rows per item = (rows of the tile) / split
    int body = -1;                              // compiled schedule of this length (-1: none)
    int body_cand = -1;                         // its index in cands (for its twiddle blocks)
    int use_body = 0;                           // 1: items run the compiled schedule
};

struct RaggedState {
    int64_t count = 0;
    int64_t total = 0;  // elements spanned by the transforms (max offset + n)
    std::vector<int64_t> n, off;
    std::vector<RaggedLenState> lens;           // one per distinct length
    int order = 1;                              // queue order: 0 = heaviest item first, 1 = grouped by length,
                                                // 2 = one sub-queue per length, home sub-queues spread over the SMs
    std::vector<RaggedItem> items;
    std::vector<long long> row_offs;
    RaggedItem* d_items = nullptr;
    long long* d_offs = nullptr;
    RaggedLen* d_lens = nullptr;
    float2* d_tw = nullptr;
    int* d_counter = nullptr;                   // one claim counter per sub-queue
    int* d_qtab = nullptr;                      // queue table (k_ragged's qtab)
    std::vector<int> qtab;
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
    if (r->d_lens) cudaFree(r->d_lens);
    if (r->d_tw) cudaFree(r->d_tw);
    if (r->d_counter) cudaFree(r->d_counter);
    if (r->d_qtab) cudaFree(r->d_qtab);
    delete r;
}

static int rows_per_item(const RaggedLenState& L) {
    const int64_t tile_rows = L.use_body ? (int64_t)kRaggedBodies[L.body].rows : (int64_t)kRaggedTile / L.n;
    const int64_t rows = tile_rows / L.split;
    return (int)std::max<int64_t>(1, std::min<int64_t>(kRaggedMaxRows, rows));
}

// Device descriptor of a length from its current schedule and pad.
static RaggedLen describe(const RaggedLenState& L) {
    RaggedLen d{};
    const std::vector<int>& sch = L.cands[L.cand];
    d.n = (int)L.n;
    d.nstages = (int)sch.size();
    d.mag_n = ragged_magic((int)L.n);
    d.body = L.use_body ? L.body : -1;
    d.tw0 = L.body_cand >= 0 ? L.tw_base[L.body_cand] : 0;
    int l = 1, tw = L.tw_base[L.cand];
    for (int s = 0; s < d.nstages; ++s) {
        RaggedStage& st = d.st[s];
        st.r = sch[s];
        st.l = l;
        st.nr = (int)L.n / sch[s];
        st.tw = tw;
        st.mag_nr = ragged_magic(st.nr);
        st.mag_l = ragged_magic(l);
        if (l > 1) tw += (sch[s] - 1) * l;
        l *= sch[s];
    }
    return d;
}

// Items from the current tile shapes: each length's transforms cut into items
// of rows_per_item rows.  Order 0: all items by work (rows * n log n),
// heaviest first (longest-processing-time list scheduling).  Order 1: items
// stay grouped by length, lengths ordered by item work, heaviest first, so
// that CTAs claiming neighbouring items run the same schedule.  Also uploads
// the length descriptors.
static gbfft_status ragged_build_items(RaggedState* r) {
    r->items.clear();
    r->row_offs.clear();
    struct Pending {
        double cost;
        int cls;
        std::vector<long long> rows;
    };
    std::vector<Pending> pend;
    const int nl = (int)r->lens.size();
    for (int c = 0; c < nl; ++c) {
        const RaggedLenState& L = r->lens[c];
        const int rows = rows_per_item(L);
        for (size_t i = 0; i < L.members.size(); i += rows) {
            Pending p;
            p.cls = c;
            const size_t e = std::min(L.members.size(), i + (size_t)rows);
            for (size_t k = i; k < e; ++k) p.rows.push_back((long long)r->off[L.members[k]]);
            p.cost = (double)p.rows.size() * L.n * std::max(1.0, std::log2((double)L.n));
            pend.push_back(std::move(p));
        }
    }
    if (r->order == 0) {
        std::stable_sort(pend.begin(), pend.end(), [](const Pending& a, const Pending& b) { return a.cost > b.cost; });
    } else {  // 1 and 2: grouped by length
        std::vector<double> cls_cost(nl, 0.0);
        for (const Pending& p : pend) cls_cost[p.cls] = std::max(cls_cost[p.cls], p.cost);
        std::stable_sort(pend.begin(), pend.end(), [&](const Pending& a, const Pending& b) {
            if (a.cls != b.cls)
                return cls_cost[a.cls] > cls_cost[b.cls] || (cls_cost[a.cls] == cls_cost[b.cls] && a.cls > b.cls);
            return a.cost > b.cost;
        });
    }
    // The last wave of the queue: items of many rows are halved, so that CTAs finish close together.
    if (r->order != 2) {
        std::vector<Pending> tail;
        const size_t k = std::min(pend.size(), (size_t)std::max(r->grid, 1));
        for (size_t i = pend.size() - k; i < pend.size(); ++i) {
            Pending& p = pend[i];
            if (p.rows.size() >= 2) {
                const size_t h = p.rows.size() / 2;
                Pending q;
                q.cls = p.cls;
                q.rows.assign(p.rows.begin() + (std::ptrdiff_t)h, p.rows.end());
                p.rows.resize(h);
                q.cost = p.cost = p.cost / 2;
                tail.push_back(std::move(q));
            }
        }
        pend.insert(pend.end(), std::make_move_iterator(tail.begin()), std::make_move_iterator(tail.end()));
    }
    for (const Pending& p : pend) {
        RaggedItem it{};
        it.cls = p.cls;
        it.count = (int)p.rows.size();
        it.first = (int)r->row_offs.size();
        it.ready = 1;
        r->items.push_back(it);
        r->row_offs.insert(r->row_offs.end(), p.rows.begin(), p.rows.end());
    }
    // Queue table: one shared queue (orders 0, 1), or one sub-queue per length in queue order (2) with
    // each SM's home sub-queue: SMs are dealt to the sub-queues in proportion to their elements (largest
    // remainder), consecutive SM ids to one sub-queue; a sub-queue too small for an SM of its own is
    // left to the CTAs that finish theirs.
    r->qtab.clear();
    if (r->order != 2 || pend.empty()) {
        r->qtab = {1, 0, 0, (int)pend.size()};
    } else {
        std::vector<int> start;
        std::vector<double> work;
        for (size_t i = 0; i < pend.size(); ++i) {
            if (i == 0 || pend[i].cls != pend[i - 1].cls) {
                start.push_back((int)i);
                work.push_back(0.0);
            }
            work.back() += (double)pend[i].rows.size() * (double)r->lens[pend[i].cls].n;
        }
        const int nq = (int)start.size();
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
            nsm = 1;
        double total = 0.0;
        for (double w : work) total += w;
        std::vector<int> sms(nq, 0);
        std::vector<std::pair<double, int>> rem;
        int dealt = 0;
        for (int k = 0; k < nq; ++k) {
            const double share = work[k] / total * nsm;
            sms[k] = (int)share;
            dealt += sms[k];
            rem.push_back({share - sms[k], k});
        }
        std::stable_sort(rem.begin(), rem.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
        for (size_t i = 0; dealt < nsm && i < rem.size(); ++i, ++dealt) ++sms[rem[i].second];
        r->qtab.push_back(nq);
        r->qtab.push_back(nsm);
        for (int k = 0; k < nq; ++k) r->qtab.push_back(start[k]);
        r->qtab.push_back((int)pend.size());
        for (int k = 0; k < nq; ++k)
            for (int i = 0; i < sms[k]; ++i) r->qtab.push_back(k);
    }
    std::vector<RaggedLen> desc(nl);
    for (int c = 0; c < nl; ++c) desc[c] = describe(r->lens[c]);
    if (r->d_qtab) cudaFree(r->d_qtab);
    r->d_qtab = nullptr;
    if (cudaMalloc(&r->d_qtab, sizeof(int) * r->qtab.size()) != cudaSuccess) {
        cudaGetLastError();
        return GBFFT_ERR_OOM;
    }
    if (cudaMemcpy(r->d_qtab, r->qtab.data(), sizeof(int) * r->qtab.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return GBFFT_ERR_CUDA;
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
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(r->d_lens, desc.data(), sizeof(RaggedLen) * nl, cudaMemcpyHostToDevice) != cudaSuccess)
        return GBFFT_ERR_CUDA;
    return GBFFT_OK;
}

static void ragged_args(RaggedState* r, const float2** pin, float2** pout, int* nitems, int** status, void** args) {
    args[0] = (void*)pin;
    args[1] = (void*)pout;
    args[2] = (void*)&r->d_items;
    args[3] = (void*)nitems;
    args[4] = (void*)&r->d_offs;
    args[5] = (void*)&r->d_lens;
    args[6] = (void*)&r->d_tw;
    args[7] = (void*)&r->d_counter;
    args[8] = (void*)&r->d_qtab;
    args[9] = (void*)status;
    args[10] = (void*)&r->wait_ns;
}

static cudaError_t ragged_launch(RaggedState* r, int direction, const void* in, void* out, int* status,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(r->d_counter, 0, sizeof(int) * (size_t)r->qtab[0], s);
    if (e != cudaSuccess) return e;
    int nitems = (int)r->items.size();
    const float2* pin = (const float2*)in;
    float2* pout = (float2*)out;
    void* args[11];
    ragged_args(r, &pin, &pout, &nitems, &status, args);
    const void* fn = direction == GBFFT_FORWARD ? ragged_kernel_fwd() : ragged_kernel_inv();
    const int grid = std::min<int>(r->grid, nitems > 0 ? nitems : 1);
    return cudaLaunchKernel(fn, dim3(grid), dim3(kRaggedThreads), args, (size_t)kRaggedSmemBytes, s);
}

gbfft_status ragged_create(RaggedState** out, const int64_t* n, const int64_t* offsets, int64_t count) {
    *out = nullptr;
    if (!n || !offsets || count < 1 || count > (int64_t)1 << 30) return GBFFT_ERR_INVALID_ARG;
    RaggedState* r = new (std::nothrow) RaggedState();
    if (!r) return GBFFT_ERR_OOM;
    r->count = count;
    r->n.assign(n, n + count);
    r->off.assign(offsets, offsets + count);
    std::vector<std::pair<int64_t, int64_t>> spans;
    spans.reserve(count);
    std::vector<int64_t> distinct;
    for (int64_t i = 0; i < count; ++i) {
        if (n[i] < 1 || offsets[i] < 0) {
            delete r;
            return GBFFT_ERR_INVALID_ARG;
        }
        if (!ragged_supported(n[i])) {
            delete r;
            return GBFFT_ERR_UNSUPPORTED_SIZE;
        }
        distinct.push_back(n[i]);
        spans.push_back({offsets[i], offsets[i] + n[i]});
        r->total = std::max(r->total, offsets[i] + n[i]);
    }
    if (r->total > ((int64_t)1 << 40)) {
        delete r;
        return GBFFT_ERR_INVALID_ARG;
    }
    std::sort(spans.begin(), spans.end());
    for (size_t i = 1; i < spans.size(); ++i) {
        if (spans[i].first < spans[i - 1].second) {
            delete r;
            return GBFFT_ERR_OVERLAP;
        }
    }
    std::sort(distinct.begin(), distinct.end());
    distinct.erase(std::unique(distinct.begin(), distinct.end()), distinct.end());
    r->lens.resize(distinct.size());
    int tw_total = 0;
    for (size_t c = 0; c < distinct.size(); ++c) {
        RaggedLenState& L = r->lens[c];
        L.n = distinct[c];
        L.cands = schedules_of(L.n);
        L.runtime_cands = (int)L.cands.size();  // a compiled schedule appended below may use composite radices
        L.body = L.n <= kRaggedMaxN ? ragged_body_id((int)L.n) : -1;
        if (L.body >= 0) {  // the compiled schedule's twiddle blocks come with the candidates
            std::vector<int> sch;
            for (int r : kRaggedBodies[L.body].radix)
                if (r > 0) sch.push_back(r);
            auto it = std::find(L.cands.begin(), L.cands.end(), sch);
            if (it == L.cands.end()) it = L.cands.insert(L.cands.end(), sch);
            L.body_cand = (int)(it - L.cands.begin());
            L.use_body = 1;
        }
        for (const auto& sch : L.cands) {
            L.tw_base.push_back(tw_total);
            tw_total += stage_twiddle_count(sch.data(), (int)sch.size());
        }
    }
    for (int64_t i = 0; i < count; ++i) {
        const size_t c = std::lower_bound(distinct.begin(), distinct.end(), n[i]) - distinct.begin();
        r->lens[c].members.push_back(i);
    }
    // Stage-twiddle blocks of every candidate schedule of every length, concatenated.
    gbfft_status st = GBFFT_OK;
    if (cudaMalloc(&r->d_tw, sizeof(float2) * (size_t)std::max(tw_total, 1)) != cudaSuccess ||
        cudaMalloc(&r->d_lens, sizeof(RaggedLen) * r->lens.size()) != cudaSuccess ||
        cudaMalloc(&r->d_counter, sizeof(int) * std::max<size_t>(distinct.size(), 1)) != cudaSuccess) {
        cudaGetLastError();
        st = GBFFT_ERR_OOM;
    }
    for (size_t c = 0; st == GBFFT_OK && c < r->lens.size(); ++c) {
        const RaggedLenState& L = r->lens[c];
        for (size_t k = 0; st == GBFFT_OK && k < L.cands.size(); ++k)
            if (launch_stage_twiddles(r->d_tw + L.tw_base[k], L.n, L.cands[k].data(), (int)L.cands[k].size(), 0) !=
                cudaSuccess)
                st = GBFFT_ERR_CUDA;
    }
    if (st == GBFFT_OK) {
        const void* ks[2] = {ragged_kernel_fwd(), ragged_kernel_inv()};
        int dev = 0, sms = 0, per_sm = 0;
        for (const void* k : ks)
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kRaggedSmemBytes) !=
                cudaSuccess)
                st = GBFFT_ERR_CUDA;
        if (st == GBFFT_OK &&
            (cudaGetDevice(&dev) != cudaSuccess ||
             cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
             cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks[0], kRaggedThreads,
                                                           (size_t)kRaggedSmemBytes) != cudaSuccess ||
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
        // kernelParams points at copies owned by the graph node; build fresh ones.
        const float2* pin = (const float2*)in;
        float2* pout = (float2*)out;
        int nitems = (int)r->items.size();
        void* args[11];
        ragged_args(r, &pin, &pout, &nitems, &status, args);
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

// Autotuner: queue order, then per length, heaviest first, the tile shape
// (rows per item = (8192/n)/split, split 1, 2, 4, 8) and the candidate radix
// schedules, by coordinate descent, timing the
// whole direct launch with CUDA events (median of `reps`).  Keeps the best
// choices and rebuilds the queue; the graph is re-captured on the next execute.
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
    // Try one setting of one knob; keep it if faster, else restore.
    auto trial = [&](int* knob, int value) {
        if (st != GBFFT_OK || *knob == value) return;
        const int keep = *knob;
        *knob = value;
        float ms = 0.f;
        st = measure(&ms);
        if (st == GBFFT_OK && ms < best) best = ms;
        else *knob = keep;
    };
    for (int o : {0, 1, 2}) trial(&r->order, o);
    std::vector<int> order;
    for (int c = 0; c < (int)r->lens.size(); ++c) order.push_back(c);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return (double)r->lens[a].members.size() * r->lens[a].n > (double)r->lens[b].members.size() * r->lens[b].n;
    });
    for (int c : order) {
        RaggedLenState& L = r->lens[c];
        if (L.body >= 0) trial(&L.use_body, 1 - L.use_body);
        const int64_t tile_rows = L.use_body ? (int64_t)kRaggedBodies[L.body].rows : (int64_t)kRaggedTile / L.n;
        for (int sp : {1, 2, 4, 8})
            if (tile_rows / sp >= 1) trial(&L.split, sp);
        if (!L.use_body)
            for (int k = 0; k < L.runtime_cands; ++k) trial(&L.cand, k);
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

gbfft_status ragged_set_queue_order(RaggedState* r, int order) {
    r->order = order;
    ragged_release_graph(r);
    return ragged_build_items(r);
}

gbfft_status ragged_set_engine(RaggedState* r, int64_t n, int compiled) {
    bool found = false;
    for (RaggedLenState& L : r->lens) {
        if (n != 0 && L.n != n) continue;
        found = true;
        if (compiled && L.body < 0) {
            if (n != 0) return GBFFT_ERR_NOT_FOUND;
            continue;  // n == 0: lengths without a compiled schedule keep the run-time engine
        }
        L.use_body = compiled ? 1 : 0;
    }
    if (!found) return GBFFT_ERR_NOT_FOUND;
    ragged_release_graph(r);
    return ragged_build_items(r);
}

int ragged_engine(const RaggedState* r, int64_t n) {
    for (const RaggedLenState& L : r->lens)
        if (L.n == n) return L.use_body;
    return -1;
}

static const RaggedLenState* len_state(const RaggedState* r, int64_t n) {
    for (const RaggedLenState& L : r->lens)
        if (L.n == n) return &L;
    return nullptr;
}

int ragged_class_split(const RaggedState* r, int64_t n) {
    const RaggedLenState* L = len_state(r, n);
    return L ? L->split : 0;
}

int ragged_schedule(const RaggedState* r, int64_t n, int* radix) {
    const RaggedLenState* L = len_state(r, n);
    if (!L) return 0;
    const std::vector<int>& sch = L->cands[L->use_body ? L->body_cand : L->cand];
    for (size_t i = 0; i < sch.size(); ++i) radix[i] = sch[i];
    return (int)sch.size();
}

bool ragged_supported(int64_t n) {
    if (n < 1 || n > kRaggedMaxN) return false;
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}


// ---------------------------------------------------------------------------
// Length table and per-call queues: ragged launches whose set of transforms
// changes from call to call (the serving loop's admission rounds).  The table
// keeps one descriptor and one schedule's twiddle blocks per length, resident
// and append-only (a kernel in flight never sees an entry change); each call
// packs its queue entries and row offsets into one blob that a single copy
// uploads, counter included.
// ---------------------------------------------------------------------------

namespace {
constexpr int kTableMaxLens = 1024;
constexpr size_t kTableTwCap = size_t(1) << 22;  // float2 entries of twiddle blocks (32 MiB)
constexpr long long kTableWaitNs = 200000000LL;  // bound on a ready-wait (every entry is published ready)
}  // namespace

struct RaggedTable {
    std::vector<RaggedLenState> lens;
    std::map<int64_t, int> cls_of;
    RaggedLen* d_lens = nullptr;
    float2* d_tw = nullptr;
    size_t tw_used = 0;
    int grid = 0;
};

void ragged_table_destroy(RaggedTable* t) {
    if (!t) return;
    if (t->d_lens) cudaFree(t->d_lens);
    if (t->d_tw) cudaFree(t->d_tw);
    delete t;
}

gbfft_status ragged_table_create(RaggedTable** out) {
    *out = nullptr;
    RaggedTable* t = new (std::nothrow) RaggedTable();
    if (!t) return GBFFT_ERR_OOM;
    if (cudaMalloc(&t->d_lens, sizeof(RaggedLen) * kTableMaxLens) != cudaSuccess ||
        cudaMalloc(&t->d_tw, sizeof(float2) * kTableTwCap) != cudaSuccess) {
        cudaGetLastError();
        ragged_table_destroy(t);
        return GBFFT_ERR_OOM;
    }
    const void* ks[2] = {ragged_kernel_fwd(), ragged_kernel_inv()};
    int dev = 0, sms = 0, per_sm = 0;
    for (const void* k : ks)
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kRaggedSmemBytes) != cudaSuccess) {
            ragged_table_destroy(t);
            return GBFFT_ERR_CUDA;
        }
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks[0], kRaggedThreads, (size_t)kRaggedSmemBytes) !=
            cudaSuccess ||
        per_sm < 1) {
        ragged_table_destroy(t);
        return GBFFT_ERR_CUDA;
    }
    t->grid = per_sm * sms;
    *out = t;
    return GBFFT_OK;
}

// The entry of length n, added (descriptor uploaded, twiddles generated on
// `s`, then synchronised) if it is new.  UNSUPPORTED_SIZE if n is not a
// 7-smooth length <= 8192, OOM if the table is full.
gbfft_status ragged_table_add(RaggedTable* t, int64_t n, cudaStream_t s, int* cls) {
    auto it = t->cls_of.find(n);
    if (it != t->cls_of.end()) {
        *cls = it->second;
        return GBFFT_OK;
    }
    if (!ragged_supported(n)) return GBFFT_ERR_UNSUPPORTED_SIZE;
    if ((int)t->lens.size() >= kTableMaxLens) return GBFFT_ERR_OOM;
    RaggedLenState L;
    L.n = n;
    std::vector<std::vector<int>> cands = schedules_of(n);
    L.body = ragged_body_id((int)n);
    std::vector<int> sch = cands.empty() ? std::vector<int>() : cands[0];
    if (L.body >= 0) {
        sch.clear();
        for (int r : kRaggedBodies[L.body].radix)
            if (r > 0) sch.push_back(r);
        L.body_cand = 0;
        L.use_body = 1;
    }
    L.cands = {sch};
    const int cnt = stage_twiddle_count(sch.data(), (int)sch.size());
    if (t->tw_used + (size_t)std::max(cnt, 1) > kTableTwCap) return GBFFT_ERR_OOM;
    L.tw_base = {(int)t->tw_used};
    const RaggedLen desc = describe(L);
    const int c = (int)t->lens.size();
    if (cnt > 0 && launch_stage_twiddles(t->d_tw + t->tw_used, n, sch.data(), (int)sch.size(), s) != cudaSuccess)
        return GBFFT_ERR_CUDA;
    if (cudaMemcpyAsync(t->d_lens + c, &desc, sizeof(RaggedLen), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GBFFT_ERR_CUDA;
    t->tw_used += (size_t)std::max(cnt, 1);
    t->lens.push_back(L);
    t->cls_of[n] = c;
    *cls = c;
    return GBFFT_OK;
}

// A queue blob starts with a 32-byte header: the claim counter (int 0) and a
// one-queue table (ints 1-4: nq = 1, no home map, the queue spanning entries
// [0, nitems)), then the entries, then the row offsets.
constexpr size_t kBlobHeader = 32;

size_t ragged_blob_bytes(int64_t nitems, int64_t nrows) {
    return kBlobHeader + sizeof(RaggedItem) * (size_t)nitems + sizeof(long long) * (size_t)nrows;
}

// Queue entries for `nspans` spans of consecutive rows (every span's length
// already in the table), heaviest entry first, packed into `blob` (at most
// `cap` bytes): the header (a zero counter and the queue table), the entries,
// the row offsets.  Returns the
// entry count, or -1 if the blob would not fit.
int64_t ragged_table_build(const RaggedTable* t, const RaggedSpan* spans, int64_t nspans, char* blob, size_t cap,
                           size_t* bytes) {
    std::vector<RaggedItem> items;
    std::vector<double> cost;
    int64_t nrows = 0;
    for (int64_t k = 0; k < nspans; ++k) {
        const RaggedLenState& L = t->lens[t->cls_of.at(spans[k].n)];
        const int64_t per = rows_per_item(L);
        for (int64_t r0 = 0; r0 < spans[k].rows; r0 += per) {
            RaggedItem it{};
            it.dout = spans[k].dout;
            it.cls = t->cls_of.at(spans[k].n);
            it.count = (int)std::min(per, spans[k].rows - r0);
            it.first = (int)(nrows + r0);
            it.ready = 1;
            items.push_back(it);
            cost.push_back((double)it.count * (double)L.n * std::max(1.0, std::log2((double)L.n)));
        }
        nrows += spans[k].rows;
    }
    const size_t need = ragged_blob_bytes((int64_t)items.size(), nrows);
    if (need > cap) return -1;
    std::vector<size_t> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    const int head[kBlobHeader / sizeof(int)] = {0, 1, 0, 0, (int)items.size(), 0, 0, 0};
    std::memcpy(blob, head, kBlobHeader);
    RaggedItem* bi = reinterpret_cast<RaggedItem*>(blob + kBlobHeader);
    for (size_t i = 0; i < order.size(); ++i) bi[i] = items[order[i]];
    long long* bo = reinterpret_cast<long long*>(blob + kBlobHeader + sizeof(RaggedItem) * items.size());
    for (int64_t k = 0, row = 0; k < nspans; ++k)
        for (int64_t r = 0; r < spans[k].rows; ++r) bo[row++] = spans[k].off + r * spans[k].n;
    *bytes = need;
    return (int64_t)items.size();
}

// One persistent launch over a blob already on the device (`d_blob`, as
// packed by ragged_table_build), transforming the rows of `data` in place.
cudaError_t ragged_table_launch(const RaggedTable* t, int direction, float2* data, const char* d_blob,
                                int64_t nitems, int* status, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    const float2* pin = data;
    float2* pout = data;
    const RaggedItem* items = reinterpret_cast<const RaggedItem*>(d_blob + kBlobHeader);
    int n_items = (int)nitems;
    const long long* offs =
        reinterpret_cast<const long long*>(d_blob + kBlobHeader + sizeof(RaggedItem) * (size_t)nitems);
    const RaggedLen* lens = t->d_lens;
    const float2* tw = t->d_tw;
    int* counter = reinterpret_cast<int*>(const_cast<char*>(d_blob));
    const int* qtab = reinterpret_cast<const int*>(d_blob) + 1;
    long long wait_ns = kTableWaitNs;
    void* args[11] = {(void*)&pin, (void*)&pout, (void*)&items,  (void*)&n_items, (void*)&offs,   (void*)&lens,
                      (void*)&tw,  (void*)&counter, (void*)&qtab, (void*)&status, (void*)&wait_ns};
    const void* fn = direction == GBFFT_FORWARD ? ragged_kernel_fwd() : ragged_kernel_inv();
    const int grid = (int)std::min<int64_t>(t->grid, nitems);
    return cudaLaunchKernel(fn, dim3(grid), dim3(kRaggedThreads), args, (size_t)kRaggedSmemBytes, s);
}

}  // namespace gbfft
