// Allocation-free form of the two-pass (Eq. 2) transform.
//
// The regular path keeps its workspace and twiddle tables in memory that
// gbfft_plan_create obtains with cudaMalloc.  Some callers cannot do that:
// hosts that own all device memory through their own fixed arena and forbid
// any further device allocation, or real-time loops (signal chains, control
// loops) that must not allocate after start-up because an allocation can
// block for an unbounded time.  gbfft_execute_twopass_noalloc serves them: it
// keeps the workspace and the tables in one file-scope device array instead,
// so the call itself allocates nothing.
//
// The array is part of this library's device image: every GPU that loads the
// library holds its kGbfftStaticScratchBytes until the process exits.  All
// calls share it and it keeps the last call's contents; nothing in it has to
// start at zero, because each call writes every table entry and every
// workspace element before reading it.  Calls that overlap on the GPU (two
// streams, or two host threads) race on the array and corrupt each other's
// results; serialise them.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "internal.h"

namespace gbfft {
namespace {

constexpr size_t kGbfftStaticScratchBytes = size_t(64) << 20;  // 64 MiB
__device__ __align__(256) unsigned char g_static_scratch[kGbfftStaticScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the array for device `dev` (current).  Host code cannot
// use the symbol itself: on the host it names a stand-in, not device memory.
cudaError_t scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

bool split_for(int64_t n, int64_t* k_out, int64_t* m_out) { return choose_split(n, 0, k_out, m_out); }

}  // namespace
}  // namespace gbfft

using namespace gbfft;

extern "C" gbfft_status gbfft_execute_twopass_noalloc(int64_t n, int64_t batch, int direction, const void* in,
                                                      void* out, void* cuda_stream) {
    if (n < 1 || batch < 0 || !in || !out) return GBFFT_ERR_INVALID_ARG;
    if (direction != GBFFT_FORWARD && direction != GBFFT_INVERSE) return GBFFT_ERR_INVALID_ARG;
    if (((uintptr_t)in & 15u) || ((uintptr_t)out & 15u)) return GBFFT_ERR_ALIGNMENT;
    int64_t k = 0, m = 0;
    if (!split_for(n, &k, &m)) return GBFFT_ERR_UNSUPPORTED_SIZE;
    const size_t bytes = sizeof(float2) * (size_t)n * (size_t)batch;
    if (in != out) {
        const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
        if (a < b + bytes && b < a + bytes) return GBFFT_ERR_OVERLAP;
    }
    const ColsVariant* cm = cols_variant_for(m);
    const ColsVariant* ck = cols_variant_for(k);
    const size_t ws_b = round256(bytes);
    const size_t post_b = round256(sizeof(float2) * (size_t)n);
    const size_t twm_b = round256(sizeof(float2) * (size_t)stage_twiddle_count(cm->radix, cm->nstages));
    const size_t twk_b = round256(sizeof(float2) * (size_t)stage_twiddle_count(ck->radix, ck->nstages));
    if (ws_b + post_b + twm_b + twk_b > kGbfftStaticScratchBytes) return GBFFT_ERR_BUDGET;
    if (batch == 0) return GBFFT_OK;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GBFFT_ERR_CUDA;
    void* base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess) return GBFFT_ERR_CUDA;
    if (prepare_cols(*cm) != cudaSuccess || prepare_cols(*ck) != cudaSuccess) return GBFFT_ERR_CUDA;

    char* p = (char*)base;
    float2* ws = (float2*)p;
    float2* post = (float2*)(p + ws_b);
    float2* tw_m = (float2*)(p + ws_b + post_b);
    float2* tw_k = (float2*)(p + ws_b + post_b + twm_b);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    bool ok = launch_post_twiddles(post, n, m, s) == cudaSuccess;
    ok = ok && launch_stage_twiddles(tw_m, m, cm->radix, cm->nstages, s) == cudaSuccess;
    ok = ok && launch_stage_twiddles(tw_k, k, ck->radix, ck->nstages, s) == cudaSuccess;
    ok = ok && launch_cols(*cm, 1, direction, (const float2*)in, ws, tw_m, post, (long long)batch, (int)k, s) ==
                   cudaSuccess;
    ok = ok && launch_cols(*ck, 2, direction, ws, (float2*)out, tw_k, nullptr, (long long)batch, (int)m, s) ==
                   cudaSuccess;
    return ok ? GBFFT_OK : GBFFT_ERR_CUDA;
}
