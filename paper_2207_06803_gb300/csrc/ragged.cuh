// Ragged batches: thousands of transforms of uneven lengths in one persistent launch.
//
// The host groups the transforms by length, gives each length a radix schedule
// (a Stockham factorisation n = R_1 ... R_t over the radices 2, 3, 4, 5, 7, 8,
// 16), cuts each group into work items of at most T rows (T * n <= 8192
// complex elements), orders the items and uploads them with the list of row
// offsets and one descriptor per length.  Each CTA of the persistent kernel
// repeatedly claims the next item with one atomic increment and runs the
// item's schedule stage by stage: the first stage reads the rows straight from
// HBM, stages exchange through a shared-memory tile, the last stage writes
// straight to HBM (the stage algebra of the single-pass kernel, Eq. 2, with
// the schedule read at run time instead of compiled per length).  Because
// only the radix is compiled (one code path per radix and stage position), a
// single kernel serves every length n <= 8192 whose prime factors are 2, 3, 5
// and 7, with a small instruction footprint and without the register pressure
// of per-length fully unrolled schedules.
//
// Items carry a `ready` word.  The host publishes all items ready; a CTA that
// claims an item still marked not ready waits for it with a bounded spin
// (globaltimer deadline), and on expiry records GBFFT_ERR_TIMEOUT in the plan's
// status word, skips the item and carries on: no wait in this kernel is
// unbounded.
#pragma once
#include <cuda_runtime.h>

#include "codelets.cuh"
#include "stockham.cuh"
#include "gbfft.h"

namespace gbfft {

constexpr int kRaggedThreads = 512;    // threads per CTA
constexpr int kRaggedTile = 8192;      // complex elements per item at most (T * n)
constexpr int kRaggedMaxRows = 512;    // rows per item at most
constexpr int kRaggedMaxStages = 8;
constexpr int kRaggedMaxN = 8192;
// Shared-memory tile with one padding slot per 16 complex (spreads the
// power-of-two strides of the exchanges across banks).
constexpr int kRaggedSmemBytes = (int)sizeof(float2) * (kRaggedTile + kRaggedTile / 16);

struct RaggedItem {
    int cls;    // index of the item's length descriptor
    int count;  // rows in this item (<= T of the length)
    int first;  // index of the item's first row offset in the offset list
    int ready;  // nonzero once the item may be processed
};

// One stage of a length's schedule: radix R, L = R_1 ... R_{s-1}, n/R
// butterflies per row, offset of the stage's twiddle block
// W[(q-1)*L + k] = w_{L R}^(q k) in the plan's table (used when L > 1), and
// the multipliers (ragged_magic) that turn the two divisions of the index
// arithmetic into one multiply-high each.
struct RaggedStage {
    int r, l, nr, tw;
    unsigned mag_nr, mag_l;
};

struct RaggedLen {
    int n, nstages;
    unsigned mag_n;
    int pad;
    RaggedStage st[kRaggedMaxStages];
};

// Division by an invariant integer with a multiply-high (the method of
// Granlund and Montgomery, 1994): with m = ceil(2^31 / d),
// floor(x / d) = floor(2x * m / 2^32) for 0 <= x < 2^31 / d.  Writing
// x = q d + r, 2x m / 2^32 = q + (r + x e / 2^31) / d with e = m d - 2^31 < d,
// and r + x e / 2^31 < d whenever x e < 2^31.  Every dividend here is below
// 8192 and every divisor at most 8192.
inline unsigned ragged_magic(int d) { return (unsigned)(((1ull << 31) + (unsigned long long)d - 1) / (unsigned)d); }

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int rdiv(int x, unsigned m) { return (int)__umulhi((unsigned)x << 1, m); }

__device__ __forceinline__ int rpad(int i) { return i + (i >> 4); }


// Butterflies of radix R per thread when the tile holds at most kRaggedTile elements.
template <int R>
constexpr int ragged_nb() {
    return (kRaggedTile / R + kRaggedThreads - 1) / kRaggedThreads;
}

// One stage on the item's `count` rows: operands from the shared tile
// (src_smem) or from the rows in HBM, results to the shared tile (dst_smem)
// or to the rows in HBM (only the last stage, where L*R = n so the write
// index b*L*R + q*L + k reduces to q*L + j).  The code is branch-free in the
// butterfly index: threads past the stage's last butterfly recompute that
// butterfly and store the same values to the same places, which keeps every
// per-butterfly guard (and the register pressure that divergent regions
// bring) out of the unrolled loops.  A duplicate may re-read an HBM row only
// in the first stage, before any stage of the item has written its output.
template <int S, int R>
__device__ __forceinline__ void ragged_stage(bool src_smem, bool dst_smem, const float2* in, float2* out,
                                             const long long* s_off, float2* sm, const float2* __restrict__ tw,
                                             const RaggedStage& st, int n, int count) {
    constexpr int NB = ragged_nb<R>();
    const int nr = st.nr, L = st.l;
    const int last = count * nr - 1;  // index of the stage's last butterfly
    const int tid = threadIdx.x;
    float2 v[NB * R];
    if (src_smem) {
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = min(tid + u * kRaggedThreads, last);
            const int t = rdiv(B, st.mag_nr), j = B - t * nr;
            const int base = t * n + j;
#pragma unroll
            for (int q = 0; q < R; ++q) v[u * R + q] = sm[rpad(base + q * nr)];
        }
    } else {
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = min(tid + u * kRaggedThreads, last);
            const int t = rdiv(B, st.mag_nr), j = B - t * nr;
            const float2* p = in + s_off[t] + j;
#pragma unroll
            for (int q = 0; q < R; ++q) v[u * R + q] = p[q * nr];
        }
    }
    if (L > 1) {
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = min(tid + u * kRaggedThreads, last);
            const int t = rdiv(B, st.mag_nr), j = B - t * nr;
            const int k = j - rdiv(j, st.mag_l) * L;
            const float2* w = tw + st.tw;
            if constexpr (R == 16) {  // four table reads, the other powers by products
                float2 p[16];
                twiddle_powers16(w, L, k, p);
#pragma unroll
                for (int q = 1; q < R; ++q) v[u * R + q] = twiddle<S>(v[u * R + q], p[q]);
            } else if constexpr (R == 8) {
                float2 p[8];
                twiddle_powers8(w, L, k, p);
#pragma unroll
                for (int q = 1; q < R; ++q) v[u * R + q] = twiddle<S>(v[u * R + q], p[q]);
            } else {
#pragma unroll
                for (int q = 1; q < R; ++q) v[u * R + q] = twiddle<S>(v[u * R + q], __ldg(w + (q - 1) * L + k));
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) Dft<S, R>::run(&v[u * R]);
    if (dst_smem) {
        if (src_smem) __syncthreads();  // every read of the tile precedes the first write
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = min(tid + u * kRaggedThreads, last);
            const int t = rdiv(B, st.mag_nr), j = B - t * nr;
            const int b = rdiv(j, st.mag_l), k = j - b * L;
            const int base = t * n + b * L * R + k;
#pragma unroll
            for (int q = 0; q < R; ++q) sm[rpad(base + q * L)] = v[u * R + q];
        }
        __syncthreads();
    } else {
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = min(tid + u * kRaggedThreads, last);
            const int t = rdiv(B, st.mag_nr), j = B - t * nr;
            float2* p = out + s_off[t] + j;
#pragma unroll
            for (int q = 0; q < R; ++q) p[q * L] = v[u * R + q];
        }
    }
}

template <int S>
__global__ void __launch_bounds__(kRaggedThreads, 2) k_ragged(const float2* in, float2* out, const RaggedItem* items,
                                                           int nitems, const long long* offs,
                                                           const RaggedLen* __restrict__ lens,
                                                           const float2* __restrict__ tw, int* counter, int* status,
                                                           long long wait_ns) {
    extern __shared__ float2 sm[];
    __shared__ long long s_off[kRaggedMaxRows];
    __shared__ RaggedLen s_len;
    __shared__ int s_item, s_ok;
    int next = 0;  // thread 0: the item claimed for the next round
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    for (;;) {
        __syncthreads();  // the previous item's readers of s_off, s_len and sm are done
        if (threadIdx.x == 0) {
            const int it = next;
            int ok = 1;
            if (it < nitems) {
                next = atomicAdd(counter, 1);  // claimed now, used next round: the latency overlaps this item
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
        {
            const int* src = reinterpret_cast<const int*>(lens + d.cls);
            int* dst = reinterpret_cast<int*>(&s_len);
            for (int w = threadIdx.x; w < (int)(sizeof(RaggedLen) / sizeof(int)); w += kRaggedThreads)
                dst[w] = __ldg(src + w);
        }
        __syncthreads();
        const int n = s_len.n, ns = s_len.nstages;
        if (ns == 0) {  // n == 1: DFT_1 is the identity
            for (int t = threadIdx.x; t < d.count; t += kRaggedThreads) out[s_off[t]] = in[s_off[t]];
            continue;
        }
        // A one-stage schedule (n <= 16) also goes through the tile, then a
        // copy writes the rows out, so that no stage reads and writes HBM.
        for (int s = 0; s < ns; ++s) {
            const RaggedStage st = s_len.st[s];
            const bool src_smem = s > 0, dst_smem = s < ns - 1 || ns == 1;
            switch (st.r) {
                case 2: ragged_stage<S, 2>(src_smem, dst_smem, in, out, s_off, sm, tw, st, n, d.count); break;
                case 3: ragged_stage<S, 3>(src_smem, dst_smem, in, out, s_off, sm, tw, st, n, d.count); break;
                case 4: ragged_stage<S, 4>(src_smem, dst_smem, in, out, s_off, sm, tw, st, n, d.count); break;
                case 5: ragged_stage<S, 5>(src_smem, dst_smem, in, out, s_off, sm, tw, st, n, d.count); break;
                case 7: ragged_stage<S, 7>(src_smem, dst_smem, in, out, s_off, sm, tw, st, n, d.count); break;
                case 8: ragged_stage<S, 8>(src_smem, dst_smem, in, out, s_off, sm, tw, st, n, d.count); break;
                case 16: ragged_stage<S, 16>(src_smem, dst_smem, in, out, s_off, sm, tw, st, n, d.count); break;
                default:
                    if (threadIdx.x == 0) atomicCAS(status, 0, (int)GBFFT_ERR_DEVICE_STATUS);
                    break;
            }
        }
        if (ns == 1) {
            const unsigned mag_n = s_len.mag_n;
            for (int idx = threadIdx.x; idx < d.count * n; idx += kRaggedThreads) {
                const int t = rdiv(idx, mag_n), j = idx - t * n;
                out[s_off[t] + j] = sm[rpad(idx)];
            }
        }
    }
}

// Kernel entry points, instantiated one direction per translation unit.
const void* ragged_kernel_fwd();
const void* ragged_kernel_inv();

}  // namespace gbfft
