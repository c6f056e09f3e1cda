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
// results; serialise them.  The array's device address is looked up in the
// current context by every call whose stream is not capturing (the address
// belongs to the context that loaded the module).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "internal.h"

namespace gbfft {
namespace {

constexpr size_t kGbfftStaticScratchBytes = size_t(64) << 20;  // 64 MiB
__device__ __align__(256) unsigned char g_static_scratch[kGbfftStaticScratchBytes];

constexpr int kMaxDevices = 64;
// Last address found per device, with the context it belongs to.  Only a call
// made while its stream is capturing uses it (see scratch_address).
struct ScratchSlot {
    CUcontext ctx = nullptr;
    void* addr = nullptr;
};
ScratchSlot g_scratch_slot[kMaxDevices];
std::mutex g_scratch_mu;

// The driver's cuCtxGetCurrent, reached through the runtime (the library does
// not link the driver library itself, so it still loads on a host without one).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn g_ctx_get_current = nullptr;

bool current_context(CUcontext* ctx) {
    if (!g_ctx_get_current) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    }
    *ctx = nullptr;
    return g_ctx_get_current(ctx) == CUDA_SUCCESS && *ctx != nullptr;
}

// Device address of the array in the current context of device `dev`.  Host
// code cannot use the symbol itself: on the host it names a stand-in, not
// device memory.  The address belongs to the context that loaded the module,
// so a call whose stream is not capturing looks it up afresh each time (a
// device reset or a different current context then cannot leave a stale
// address behind); a call whose stream is capturing reuses the address the
// last uncaptured call found in the same context, and fails if there is none.
cudaError_t scratch_address(int dev, cudaStream_t s, void** out) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchSlot& slot = g_scratch_slot[dev];
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        CUcontext ctx = nullptr;
        if (!current_context(&ctx)) return cudaErrorDeviceUninitialized;
        slot.ctx = ctx;
        slot.addr = p;
        *out = p;
        return cudaSuccess;
    }
    CUcontext ctx = nullptr;
    if (!current_context(&ctx) || ctx != slot.ctx || !slot.addr)
        return cudaErrorDeviceUninitialized;
    *out = slot.addr;
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
    // Bound batch before multiplying, so that the byte count cannot wrap.
    if (batch > (int64_t)(kGbfftStaticScratchBytes / (sizeof(float2) * (size_t)n))) return GBFFT_ERR_BUDGET;
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
    if (scratch_address(dev, (cudaStream_t)cuda_stream, &base) != cudaSuccess) return GBFFT_ERR_CUDA;
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
