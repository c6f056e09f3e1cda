// Ragged batches: thousands of transforms of uneven lengths in one persistent launch.
//
// The host groups the transforms by length ("class"), cuts each group into
// work items of at most T_c rows (the tile shape of class c, chosen by the
// autotuner), orders the items longest-first and uploads them with the list of
// row offsets.  Each CTA of the persistent kernel repeatedly claims the next
// item with one atomic increment and runs the class's Stockham schedule on it
// (the same stage code as the single-pass kernel, with per-row offsets held in
// shared memory), until the queue is empty.  Every class uses 256 threads per
// CTA, so one kernel serves all classes.
//
// Items carry a `ready` word.  The host publishes all items ready; a CTA that
// claims an item still marked not ready waits for it with a bounded spin
// (globaltimer deadline), and on expiry records GBFFT_ERR_TIMEOUT in the plan's
// status word, skips the item and carries on: no wait in this kernel is
// unbounded.
#pragma once
#include <cuda_runtime.h>

#include "gbfft.h"
#include "stockham.cuh"

namespace gbfft {

constexpr int kRaggedThreads = 256;

struct RaggedItem {
    int cls;    // class index (length) in the class table
    int count;  // rows in this item (<= T of the class)
    int first;  // index of the item's first row offset in the offset list
    int ready;  // nonzero once the item may be processed
};

// (case index, N, T rows per full tile, shared-memory pad shift, radix
// schedule...).  Every class runs kRaggedThreads threads; T is about
// 4096/N (at most 256) so a tile holds ~4096 elements and each thread at most
// 32 complex values; a stage with fewer butterflies than threads leaves some
// idle.
#define GBFFT_RAGGED_CLASSES(X)               \
    X(0, 8, 256, 4, 2, 4)                     \
    X(1, 10, 256, 0, 5, 2)                    \
    X(2, 12, 256, 0, 3, 4)                    \
    X(3, 14, 256, 0, 7, 2)                    \
    X(4, 16, 256, 4, 4, 4)                    \
    X(5, 20, 204, 0, 5, 4)                    \
    X(6, 24, 170, 0, 3, 8)                    \
    X(7, 28, 146, 0, 7, 4)                    \
    X(8, 32, 128, 4, 4, 8)                    \
    X(9, 40, 102, 0, 5, 8)                    \
    X(10, 48, 85, 4, 3, 16)                   \
    X(11, 56, 73, 0, 7, 8)                    \
    X(12, 64, 64, 4, 8, 8)                    \
    X(13, 80, 51, 5, 5, 16)                   \
    X(14, 96, 42, 4, 3, 2, 16)                \
    X(15, 112, 36, 4, 7, 16)                  \
    X(16, 128, 32, 4, 8, 16)                  \
    X(17, 160, 25, 0, 5, 2, 16)               \
    X(18, 192, 21, 0, 3, 4, 16)               \
    X(19, 224, 18, 0, 7, 2, 16)               \
    X(20, 256, 16, 4, 16, 16)                 \
    X(21, 320, 12, 0, 5, 4, 16)               \
    X(22, 384, 10, 0, 3, 8, 16)               \
    X(23, 448, 9, 0, 7, 4, 16)                \
    X(24, 512, 8, 4, 2, 16, 16)               \
    X(25, 640, 6, 0, 5, 8, 16)                \
    X(26, 768, 5, 4, 3, 16, 16)               \
    X(27, 896, 4, 0, 7, 8, 16)                \
    X(28, 1024, 4, 4, 4, 16, 16)              \
    X(29, 1280, 3, 5, 5, 16, 16)              \
    X(30, 1536, 2, 4, 3, 16, 16, 2)           \
    X(31, 1792, 2, 4, 7, 16, 16)              \
    X(32, 2048, 2, 4, 16, 16, 8)              \
    X(33, 2560, 1, 5, 5, 16, 16, 2)           \
    X(34, 3072, 1, 4, 3, 16, 16, 4)           \
    X(35, 3584, 1, 4, 7, 16, 16, 2)           \
    X(36, 4096, 1, 4, 16, 16, 16)             \
    X(37, 5120, 1, 4, 5, 16, 16, 4)           \
    X(38, 6144, 1, 4, 3, 16, 16, 8)           \
    X(39, 7168, 1, 4, 7, 16, 16, 4)           \
    X(40, 8192, 1, 4, 16, 16, 32)             \
    X(41, 256, 16, 4, 4, 8, 8)                \
    X(42, 512, 8, 4, 8, 8, 8)                 \
    X(43, 1024, 4, 4, 16, 16, 4)              \
    X(44, 2048, 2, 4, 8, 16, 16)              \
    X(45, 4096, 1, 4, 8, 8, 8, 8)             \
    X(46, 8192, 1, 4, 16, 16, 16, 2)          \
    X(47, 3072, 1, 4, 3, 8, 8, 8, 2)          \
    X(48, 128, 32, 4, 2, 8, 8)                \
    X(49, 20, 102, 0, 5, 4)                   \
    X(50, 24, 85, 0, 3, 8)                    \
    X(51, 28, 73, 0, 7, 4)                    \
    X(52, 40, 51, 0, 5, 8)                    \
    X(53, 48, 42, 4, 3, 16)                   \
    X(54, 56, 36, 0, 7, 8)                    \
    X(55, 80, 25, 5, 5, 16)                   \
    X(56, 96, 21, 4, 3, 2, 16)                \
    X(57, 112, 18, 4, 7, 16)                  \
    X(58, 160, 12, 0, 5, 2, 16)               \
    X(59, 192, 10, 0, 3, 4, 16)               \
    X(60, 224, 9, 0, 7, 2, 16)                \
    X(61, 448, 4, 0, 7, 4, 16)

// Compiled cases: the first case of each length (indices 0..40) is its default
// schedule; cases 41.. are alternatives the autotuner may choose: other radix
// schedules (41-48) and half-height tiles, whose smaller per-thread register
// arrays avoid spills for the odd-radix lengths (49-61).
constexpr int kRaggedCases = 62;


__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int S, int N, int T, int PS, int... Rs>
__device__ __noinline__ void ragged_item(const float2* in, float2* out, const long long* s_off, float2* sm,
                                            const float2* __restrict__ tw, int nvalid) {
    constexpr int TPB = kRaggedThreads;
    constexpr int E = capacity_of_r<N, T, TPB, Rs...>();
    static_assert(T >= 1 && T <= kRaggedThreads && E <= 32, "class tile shape");
    const IndexedIO<N> io{in, out, s_off};
    float2 v[E];
    gather_global<N, E, T, First<Rs...>::value, IndexedIO<N>, TPB>(v, io, nvalid);
    run_stages_t<N, S, E, T, PS, TPB, true, 0, 1, Rs...>(v, io, sm, tw, nvalid);
}

template <int S>
__global__ void __launch_bounds__(kRaggedThreads, 3) k_ragged(const float2* in, float2* out, const RaggedItem* items,
                                                           int nitems, const long long* offs,
                                                           const float2* __restrict__ tw,
                                                           const int* __restrict__ tw_off, int* counter, int* status,
                                                           long long wait_ns) {
    extern __shared__ float2 sm[];
    __shared__ long long s_off[kRaggedThreads];
    __shared__ int s_item, s_ok;
    for (;;) {
        __syncthreads();  // the previous item's readers of s_off and sm are done
        if (threadIdx.x == 0) {
            const int it = atomicAdd(counter, 1);
            int ok = 1;
            if (it < nitems) {
                const volatile int* rdy = &items[it].ready;
                if (*rdy == 0) {
                    const unsigned long long t0 = globaltimer_ns();
                    while (*rdy == 0) {
                        if (globaltimer_ns() - t0 > (unsigned long long)wait_ns) {
                            ok = 0;
                            atomicCAS(status, 0, (int)GBFFT_ERR_TIMEOUT);
                            break;
                        }
                        __nanosleep(2000);
                    }
                }
            }
            s_item = it;
            s_ok = ok;
        }
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        if (!s_ok) continue;
        const RaggedItem d = items[it];
        for (int t = threadIdx.x; t < d.count; t += kRaggedThreads) s_off[t] = offs[d.first + t];
        __syncthreads();
        const float2* twc = tw + tw_off[d.cls];
        switch (d.cls) {
#define GBFFT_RAGGED_CASE(idx, N, T, PS, ...)                                      \
    case idx:                                                                     \
        ragged_item<S, N, T, PS, __VA_ARGS__>(in, out, s_off, sm, twc, d.count); \
        break;
            GBFFT_RAGGED_CLASSES(GBFFT_RAGGED_CASE)
#undef GBFFT_RAGGED_CASE
            default:
                if (threadIdx.x == 0) atomicCAS(status, 0, (int)GBFFT_ERR_DEVICE_STATUS);
                break;
        }
    }
}

// Kernel entry points, instantiated one direction per translation unit.
const void* ragged_kernel_fwd();
const void* ragged_kernel_inv();

}  // namespace gbfft
