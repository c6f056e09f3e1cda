// Ragged batches: thousands of transforms of uneven lengths in one persistent launch.
//
// The host groups the transforms by length, gives each length a radix schedule
// (a Stockham factorisation n = R_1 ... R_t), cuts each group into work items
// of at most T rows (T * n <= 8192 complex elements), orders the items and
// uploads them with the list of row offsets and one descriptor per length.
// Each CTA of the persistent kernel repeatedly claims queue items (one atomic
// per item, from a shared queue or from per-length sub-queues with a home
// sub-queue per SM) and runs each item's schedule: the first stage reads the
// rows straight from HBM, stages exchange through a shared-memory tile, the last
// stage writes straight to HBM (the stage algebra of the single-pass kernel,
// Eq. 2).  Two engines run a schedule:
//   compiled  for n = p * 2^k (p = 1, 3, 5, 7, 8 <= n <= 8192): the schedule
//             and the tile are fixed at compile time, one non-inlined function
//             per length with its own register allocation (constant strides
//             fold into addressing: a third fewer instructions than the
//             run-time engine on the 41-length mix);
//   run-time  any n <= 8192 whose prime factors are 2, 3, 5, 7: the schedule is
//             read from the length's descriptor, one code path per radix.
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
    int cls;         // index of the item's length descriptor
    int count;       // rows in this item (<= T of the length)
    int first;       // index of the item's first row offset in the offset list
    int ready;       // nonzero once the item may be processed
    long long dout;  // the item's output rows start dout complex elements after its input rows' offsets
    long long pad;
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
    int body;  // compiled schedule (index into the body list below), or -1: the run-time stage engine
    int tw0;   // offset of the compiled schedule's stage-twiddle blocks in the plan's table
    int pad[3];
    RaggedStage st[kRaggedMaxStages];
};
static_assert(sizeof(RaggedLen) % 16 == 0, "descriptors are copied in 16-byte pieces");
constexpr int kRaggedLenChunks = (int)(sizeof(RaggedLen) / 16);
static_assert(sizeof(RaggedItem) == 32, "queue entries are copied in two 16-byte pieces");

// Compiled schedules.  For the lengths n = p * 2^k (p = 1, 3, 5, 7, 8 <= n <=
// 8192) an item runs a schedule fixed at compile time: the single-pass stage
// engine of stockham.cuh with constant strides, so index arithmetic folds into
// addressing and the twiddle loop bounds are known.  X(N, T, radices...): T
// rows per item (T * N <= 8192 elements; for p = 3, 5, 7 the tile is capped so
// that the first stage holds at most 16 complex per thread where it can),
// radices in application order.  The first stage carries the odd factor: a
// lone radix p, or a composite p * 2^j (DFT_6 ... DFT_28, prime-factor
// codelets) where that saves a fourth stage or an uneven radix-2/4 stage.
// Every other 7-smooth length runs the run-time engine (radices 2 ... 16).
#define GBFFT_RAGGED_BODIES(X)   \
    X(8, 512, 2, 4)              \
    X(16, 512, 4, 4)             \
    X(32, 256, 4, 8)             \
    X(64, 128, 4, 16)            \
    X(128, 64, 8, 16)            \
    X(256, 32, 16, 16)           \
    X(512, 16, 2, 16, 16)        \
    X(1024, 8, 4, 16, 16)        \
    X(2048, 4, 16, 16, 8)        \
    X(4096, 2, 16, 16, 16)       \
    X(8192, 1, 16, 16, 16, 2)    \
    X(12, 512, 3, 4)             \
    X(24, 320, 3, 8)             \
    X(48, 160, 3, 16)            \
    X(96, 64, 6, 16)             \
    X(192, 32, 12, 16)           \
    X(384, 20, 3, 8, 16)         \
    X(768, 10, 3, 16, 16)        \
    X(1536, 4, 6, 16, 16)        \
    X(3072, 2, 12, 16, 16)       \
    X(6144, 1, 3, 16, 16, 8)     \
    X(10, 512, 5, 2)             \
    X(20, 384, 5, 4)             \
    X(40, 192, 5, 8)             \
    X(80, 96, 5, 16)             \
    X(160, 32, 10, 16)           \
    X(320, 24, 5, 4, 16)         \
    X(640, 12, 5, 8, 16)         \
    X(1280, 6, 5, 16, 16)        \
    X(2560, 2, 10, 16, 16)       \
    X(5120, 1, 5, 16, 16, 4)     \
    X(14, 512, 7, 2)             \
    X(28, 256, 7, 4)             \
    X(56, 128, 7, 8)             \
    X(112, 64, 7, 16)            \
    X(224, 32, 14, 16)           \
    X(448, 16, 7, 4, 16)         \
    X(896, 8, 7, 8, 16)          \
    X(1792, 4, 7, 16, 16)        \
    X(3584, 2, 14, 16, 16)       \
    X(7168, 1, 7, 16, 16, 4)

// Host-side description of a compiled schedule (plan building, autotuner).
struct RaggedBodyInfo {
    int n, rows;
    int radix[kRaggedMaxStages];
};
#define GBFFT_RAGGED_BODY_INFO(N, T, ...) {N, T, {__VA_ARGS__}},
constexpr RaggedBodyInfo kRaggedBodies[] = {GBFFT_RAGGED_BODIES(GBFFT_RAGGED_BODY_INFO)};
#undef GBFFT_RAGGED_BODY_INFO
constexpr int kRaggedNumBodies = (int)(sizeof(kRaggedBodies) / sizeof(kRaggedBodies[0]));

constexpr int ragged_body_id(int n) {
    for (int i = 0; i < kRaggedNumBodies; ++i)
        if (kRaggedBodies[i].n == n) return i;
    return -1;
}

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

// Rows of an item: row t starts at complex element off[t] of both buffers
// (the offsets stay in global memory, read once per butterfly through the
// read-only path).
struct RaggedIO {
    const float2* in;
    float2* out;
    const long long* __restrict__ off;
    __device__ __forceinline__ float2 ld(int t, int n) const { return in[off[t] + n]; }
    __device__ __forceinline__ void st(int t, int n, float2 v) const { out[off[t] + n] = v; }
};

// One item on a compiled schedule: stage 1 reads the rows from HBM, stages
// exchange through the padded tile, the last stage writes HBM; rows t >=
// nvalid of the T-row tile are skipped.  The caller has synchronised since
// the tile's last readers.
template <int N, int S, int T, int... Rs>
__device__ __noinline__ void ragged_body(const float2* in, float2* out, const long long* __restrict__ off, float2* sm,
                                         const float2* __restrict__ tw, int nvalid) {
    constexpr int E = capacity_of_r<N, T, kRaggedThreads, Rs...>();
    static_assert(T * N <= kRaggedTile && E <= 16, "compiled ragged tile too large");
    float2 v[E];
    const RaggedIO io{in, out, off};
    gather_global<N, E, T, First<Rs...>::value, RaggedIO, kRaggedThreads>(v, io, nvalid);
    run_stages_t<N, S, E, T, 4, kRaggedThreads, false, 0, 1, Rs...>(v, io, sm, tw, nvalid);
}

template <int S>
__device__ __forceinline__ void ragged_compiled(int body, const float2* in, float2* out, const long long* off,
                                                float2* sm, const float2* __restrict__ tw, int nvalid) {
    switch (body) {
#define GBFFT_RAGGED_BODY_CASE(N, T, ...)                          \
    case ragged_body_id(N):                                        \
        ragged_body<N, S, T, __VA_ARGS__>(in, out, off, sm, tw, nvalid);     \
        break;
        GBFFT_RAGGED_BODIES(GBFFT_RAGGED_BODY_CASE)
#undef GBFFT_RAGGED_BODY_CASE
        default:
            break;
    }
}

// Asynchronous global -> shared copies (cp.async): complete per thread at
// ragged_cp_async_wait, visible to the CTA after the next barrier.
__device__ __forceinline__ void ragged_cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void ragged_cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void ragged_cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The queue is cut into nq sub-queues (consecutive ranges of entries), each
// with its own claim counter.  Queue table `qtab`: qtab[0] = nq, qtab[1] =
// nhome, qtab[2 ... 2+nq] = the entry index where each sub-queue starts (the
// last = nitems), then nhome entries giving the sub-queue each SM (by %smid)
// starts on.  Thread 0 claims one entry at a time from its current sub-queue
// and, when that sub-queue is exhausted, moves on to the next one in ring
// order: sub-queues never refill, so each CTA visits every sub-queue at most
// once after its home and issues at most nq failing claims in all.  With one
// sub-queue and no home map this is a single shared queue.  With one
// sub-queue per length and home sub-queues spread over the SMs in proportion
// to each length's work, an SM runs few distinct lengths: their compiled code
// and stage twiddles stay in its caches.
template <int S>
__global__ void __launch_bounds__(kRaggedThreads, 2) k_ragged(const float2* in, float2* out, const RaggedItem* items,
                                                           int nitems, const long long* offs,
                                                           const RaggedLen* __restrict__ lens,
                                                           const float2* __restrict__ tw, int* counters,
                                                           const int* __restrict__ qtab, int* status,
                                                           long long wait_ns) {
    extern __shared__ float2 sm[];
    __shared__ __align__(16) long long s_off[2][kRaggedMaxRows];
    __shared__ __align__(16) RaggedLen s_len[2];
    __shared__ __align__(16) RaggedItem s_item[3];
    __shared__ int s_id[3];
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    // Descriptor and row offsets of queue entry d into descriptor slot ls (every thread).
    auto fetch = [&](const RaggedItem& d, int ls) {
        if (tid < kRaggedLenChunks)
            ragged_cp_async16(reinterpret_cast<char*>(&s_len[ls]) + 16 * tid,
                              reinterpret_cast<const char*>(lens + d.cls) + 16 * tid);
        for (int t = tid; t < d.count; t += kRaggedThreads) ragged_cp_async8(&s_off[ls][t], offs + d.first + t);
    };
    int q = 0, nq = 1, left = 0;  // thread 0: current sub-queue, sub-queue count, sub-queues not yet found empty
    const int* qstart = qtab + 2;
    auto claim = [&]() {  // thread 0: the next queue index, nitems once every sub-queue is exhausted
        while (left > 0) {
            const int idx = qstart[q] + atomicAdd(&counters[q], 1);
            if (idx < qstart[q + 1]) return idx;
            q = q + 1 == nq ? 0 : q + 1;
            --left;
        }
        return nitems;
    };
    if (tid == 0) {
        nq = qtab[0];
        left = nq;
        const int nhome = qtab[1];
        if (nhome > 0) {
            unsigned smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            q = (int)smid < nhome ? qtab[3 + nq + smid] : 0;
        }
        for (int k = 0; k < 2; ++k) {
            const int id = claim();
            s_id[k] = id;
            if (id < nitems) {
                ragged_cp_async16(&s_item[k], items + id);
                ragged_cp_async16(reinterpret_cast<char*>(&s_item[k]) + 16, reinterpret_cast<const char*>(items + id) + 16);
            }
        }
        ragged_cp_async_wait();
    }
    __syncthreads();
    if (s_id[0] < nitems) fetch(s_item[0], 0);
    for (int i = 0;; ++i) {
        const int cur = i % 3, nxt = (i + 1) % 3, aft = (i + 2) % 3, ls = i & 1;
        if (tid == 0) {  // this item's entry was read an item ago; wait (bounded) if it was not ready then
            int ok = 1;
            const int it = s_id[cur];
            if (it < nitems && s_item[cur].ready == 0) {
                const volatile int* rdy = &items[it].ready;
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
            s_ok = ok;
        }
        ragged_cp_async_wait();  // this thread's copies of the item's descriptor and offsets
        __syncthreads();         // the previous item's readers of the tile and of the other slot are done
        const int it = s_id[cur];
        if (it >= nitems) break;
        const int count = s_item[cur].count;
        float2* const iout = out + s_item[cur].dout;  // this item's output rows (off[t] from here)
        if (s_id[nxt] < nitems) fetch(s_item[nxt], ls ^ 1);
        if (tid == 0) {
            const int id = claim();
            s_id[aft] = id;
            if (id < nitems) {
                ragged_cp_async16(&s_item[aft], items + id);
                ragged_cp_async16(reinterpret_cast<char*>(&s_item[aft]) + 16,
                                  reinterpret_cast<const char*>(items + id) + 16);
            }
        }
        if (!s_ok) continue;
        const long long* off = s_off[ls];
        const int body = s_len[ls].body;
        if (body >= 0) {
            ragged_compiled<S>(body, in, iout, off, sm, tw + s_len[ls].tw0, count);
            continue;
        }
        const int n = s_len[ls].n, ns = s_len[ls].nstages;
        if (ns == 0) {  // n == 1: DFT_1 is the identity
            for (int t = tid; t < count; t += kRaggedThreads) iout[off[t]] = in[off[t]];
            continue;
        }
        // A one-stage schedule (n <= 16) also goes through the tile, then a
        // copy writes the rows out, so that no stage reads and writes HBM.
        for (int s = 0; s < ns; ++s) {
            const RaggedStage st = s_len[ls].st[s];
            const bool src_smem = s > 0, dst_smem = s < ns - 1 || ns == 1;
            switch (st.r) {
                case 2: ragged_stage<S, 2>(src_smem, dst_smem, in, iout, off, sm, tw, st, n, count); break;
                case 3: ragged_stage<S, 3>(src_smem, dst_smem, in, iout, off, sm, tw, st, n, count); break;
                case 4: ragged_stage<S, 4>(src_smem, dst_smem, in, iout, off, sm, tw, st, n, count); break;
                case 5: ragged_stage<S, 5>(src_smem, dst_smem, in, iout, off, sm, tw, st, n, count); break;
                case 7: ragged_stage<S, 7>(src_smem, dst_smem, in, iout, off, sm, tw, st, n, count); break;
                case 8: ragged_stage<S, 8>(src_smem, dst_smem, in, iout, off, sm, tw, st, n, count); break;
                case 16: ragged_stage<S, 16>(src_smem, dst_smem, in, iout, off, sm, tw, st, n, count); break;
                default:
                    if (tid == 0) atomicCAS(status, 0, (int)GBFFT_ERR_DEVICE_STATUS);
                    break;
            }
        }
        if (ns == 1) {
            const unsigned mag_n = s_len[ls].mag_n;
            for (int idx = tid; idx < count * n; idx += kRaggedThreads) {
                const int t = rdiv(idx, mag_n), j = idx - t * n;
                iout[off[t] + j] = sm[rpad(idx)];
            }
        }
    }
}

// Kernel entry points, instantiated one direction per translation unit.
const void* ragged_kernel_fwd();
const void* ragged_kernel_inv();

}  // namespace gbfft
