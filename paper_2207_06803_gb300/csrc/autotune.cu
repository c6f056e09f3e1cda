// Planner autotuner and wisdom (the planner the paper lists as future work,
// in the spirit of FFTW's runtime planner, Sec. III).
//
// gbfft_autotune times every way this library can run one length - each
// compiled single-pass variant (radix schedule x tile shape x kernel shape),
// each Eq. 2 two-pass split N = K * M, each tensor-core engine, each FP64
// variant of a complex128 plan - on scratch
// buffers of the requested batch, and records the fastest in an in-process
// wisdom table keyed by (n, dtype, direction).  gbfft_plan_create consults the
// table when no variant is forced.  Wisdom is saved to / loaded from a text
// file, one entry per line:
//     gbfft-wisdom 1 <gpu name with '_' for spaces> <n> <dtype> <direction> <variant> <k_outer> <ms>
// Entries measured on another GPU model are skipped on load.  If the
// environment variable GBFFT_WISDOM names a file, it is loaded once, at the
// first plan creation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace gbfft {
namespace {

struct Wisdom {
    int variant;      // single-pass variant index or tensor-core engine; -1 with k_outer > 0 = two-pass
    int64_t k_outer;  // > 0: two-pass split
    float ms;
};

std::mutex g_mu;
std::map<std::tuple<int64_t, int, int>, Wisdom> g_wisdom;
bool g_env_loaded = false;

std::string gpu_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string s = prop.name;
    for (char& c : s)
        if (c == ' ' || c == '\t') c = '_';
    return s;
}

gbfft_status load_file(const char* path, bool require_gpu_match) {
    FILE* f = std::fopen(path, "r");
    if (!f) return GBFFT_ERR_NOT_FOUND;
    const std::string me = require_gpu_match ? gpu_name() : std::string();
    char tag[32], name[256];
    int ver = 0, dtype = 0, dir = 0, variant = 0;
    long long n = 0, k = 0;
    float ms = 0;
    gbfft_status st = GBFFT_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    while (true) {
        const int got = std::fscanf(f, "%31s %d %255s %lld %d %d %d %lld %f", tag, &ver, name, &n, &dtype, &dir,
                                    &variant, &k, &ms);
        if (got == EOF) break;
        if (got != 9 || std::strcmp(tag, "gbfft-wisdom") != 0 || ver != 1) {
            st = GBFFT_ERR_INVALID_ARG;
            break;
        }
        if (require_gpu_match && me != name) continue;
        g_wisdom[std::make_tuple((int64_t)n, dtype, dir)] = Wisdom{variant, (int64_t)k, ms};
    }
    std::fclose(f);
    return st;
}

float time_plan(gbfft_plan p, const void* in, void* out, int reps, cudaStream_t s) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> t;
    for (int i = 0; i < reps + 2; ++i) {
        cudaEventRecord(e0, s);
        if (gbfft_execute(p, in, out, s) != GBFFT_OK) {
            t.clear();
            break;
        }
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            t.clear();
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (i >= 2) t.push_back(ms);  // two warm-up runs
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (t.empty()) return -1.f;
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

}  // namespace

void wisdom_load_env_once() {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_env_loaded) return;
        g_env_loaded = true;
    }
    const char* path = std::getenv("GBFFT_WISDOM");
    if (path && *path) load_file(path, true);
}

bool wisdom_lookup(int64_t n, int dtype, int direction, int* variant, int64_t* k_outer) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_wisdom.find(std::make_tuple(n, dtype, direction));
    if (it == g_wisdom.end()) return false;
    *variant = it->second.variant;
    *k_outer = it->second.k_outer;
    return true;
}

}  // namespace gbfft

using namespace gbfft;

extern "C" {

gbfft_status gbfft_autotune(int64_t n, int64_t batch, int direction, int dtype, int reps, int* best_variant,
                            int64_t* best_k_outer, float* best_ms) {
    if (n < 1 || batch < 1 || reps < 1) return GBFFT_ERR_INVALID_ARG;
    if (direction != GBFFT_FORWARD && direction != GBFFT_INVERSE) return GBFFT_ERR_INVALID_ARG;
    struct Cand {
        int variant;
        int64_t k;
    };
    std::vector<Cand> cands;
    if (dtype == GBFFT_C2C_F32) {
        const int nv = gbfft_num_variants(n);
        for (int v = 0; v < nv; ++v) cands.push_back({v, 0});
        static const int64_t lens[] = {32, 48, 64, 80, 96, 112, 128, 256, 512};
        for (int64_t k : lens)
            if (n % k == 0 && (n / k) % 16 == 0 && cols_variant_for(k) && cols_variant_for(n / k))
                cands.push_back({-1, k});
    } else if (dtype == GBFFT_C2C_F64) {
        const int nv = rows_variants_f64_for(n, nullptr, 0);
        for (int v = 0; v < nv; ++v) cands.push_back({v, 0});
    } else if (dtype == GBFFT_C2C_F32_TC_FP16X2 || dtype == GBFFT_C2C_F32_TC_BF16X2) {
        for (int e = 0; e < 4; ++e) cands.push_back({e, 0});  // mma.sync, tcgen05 Stockham, direct DFT (2 forms)
    } else {
        return GBFFT_ERR_INVALID_ARG;
    }
    if (cands.empty()) return GBFFT_ERR_UNSUPPORTED_SIZE;
    const size_t bytes = (dtype == GBFFT_C2C_F64 ? sizeof(double2) : sizeof(float2)) * (size_t)n * (size_t)batch;
    void *din = nullptr, *dout = nullptr;
    if (cudaMalloc(&din, bytes) != cudaSuccess || cudaMalloc(&dout, bytes) != cudaSuccess) {
        cudaGetLastError();
        if (din) cudaFree(din);
        return GBFFT_ERR_OOM;
    }
    cudaMemset(din, 0, bytes);
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    float best = -1.f;
    Cand pick{-1, 0};
    for (const Cand& c : cands) {
        gbfft_plan p = nullptr;
        gbfft_status st = c.k > 0 ? gbfft_plan_create_twopass(&p, n, batch, direction, dtype, c.k)
                                  : gbfft_plan_create_variant(&p, n, batch, direction, dtype, c.variant);
        if (st != GBFFT_OK) continue;  // e.g. an engine this length does not have
        const float ms = time_plan(p, din, dout, reps, s);
        gbfft_destroy(p);
        if (ms > 0.f && (best < 0.f || ms < best)) {
            best = ms;
            pick = c;
        }
    }
    cudaStreamDestroy(s);
    cudaFree(din);
    cudaFree(dout);
    if (best < 0.f) return GBFFT_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_wisdom[std::make_tuple(n, dtype, direction)] = Wisdom{pick.variant, pick.k, best};
    }
    if (best_variant) *best_variant = pick.variant;
    if (best_k_outer) *best_k_outer = pick.k;
    if (best_ms) *best_ms = best;
    return GBFFT_OK;
}

gbfft_status gbfft_wisdom_lookup(int64_t n, int dtype, int direction, int* variant, int64_t* k_outer) {
    int v = 0;
    int64_t k = 0;
    if (!wisdom_lookup(n, dtype, direction, &v, &k)) return GBFFT_ERR_NOT_FOUND;
    if (variant) *variant = v;
    if (k_outer) *k_outer = k;
    return GBFFT_OK;
}

gbfft_status gbfft_wisdom_export(const char* path) {
    if (!path) return GBFFT_ERR_INVALID_ARG;
    FILE* f = std::fopen(path, "w");
    if (!f) return GBFFT_ERR_INVALID_ARG;
    const std::string name = gpu_name();
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& kv : g_wisdom)
        std::fprintf(f, "gbfft-wisdom 1 %s %lld %d %d %d %lld %.6f\n", name.c_str(), (long long)std::get<0>(kv.first),
                     std::get<1>(kv.first), std::get<2>(kv.first), kv.second.variant, (long long)kv.second.k_outer,
                     kv.second.ms);
    std::fclose(f);
    return GBFFT_OK;
}

gbfft_status gbfft_wisdom_import(const char* path, int require_same_gpu) {
    if (!path) return GBFFT_ERR_INVALID_ARG;
    return load_file(path, require_same_gpu != 0);
}

gbfft_status gbfft_wisdom_forget(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_wisdom.clear();
    return GBFFT_OK;
}

}  // extern "C"
