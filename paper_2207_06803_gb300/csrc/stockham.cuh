// Single-pass Stockham engine: one CTA transforms T contiguous rows of length N.
//
// Schedule N = R_1 * R_2 * ... * R_t.  Stage s has radix R = R_s,
// L = R_1 * ... * R_{s-1} (L = 1 at s = 1) and L' = L * R.  Butterfly j < N/R of
// a row, written j = b*L + k (k < L), reads
//     a_q = x[j + q*N/R] * w_{L'}^(q*k),      q < R
// computes A = DFT_R a in registers and writes
//     y[b*L' + q*L + k] = A_q.
// In matrix form a stage is (Pi (x) I_L) (DFT_R (x) I_{N/R}) D, the factor types
// of Eq. 2 (Kronecker product with an identity, twiddle diagonal, stride
// permutation), and DFT_N = S_t ... S_1 with the output in natural order (the
// self-sorting Stockham arrangement).  The permutation is never a pass over
// memory: it is the address pattern of the write into shared memory.
//
// Data movement per CTA: the first stage reads its operands straight from HBM
// (for each q, consecutive threads read consecutive elements of a row), the
// stages exchange through shared memory, and the last stage writes straight to
// HBM (again consecutive threads, consecutive elements).  Twiddles come from
// per-plan stage tables (FP64-generated, stored as float2): for every stage
// with L > 1, the (R-1) x L block W_s[q-1][k] = w_{L'}^(q*k) = w_N^(q*k*N/L'),
// stored q-major so that consecutive threads (consecutive k) read consecutive
// entries; the blocks of successive stages are concatenated.  The inverse
// uses the conjugate.  FP32 radix-16 stages read only q = 1, 2, 4, 8 and form
// the other powers by products.
//
// Three kernel shapes share the stage code:
//   k_stockham_rows     one tile per CTA, grid = number of tiles;
//   k_stockham_rows_pf  persistent: grid = resident CTAs, each CTA walks tiles
//                       and issues the HBM loads of its next tile before it
//                       computes the current one (register prefetch), so the
//                       loads overlap the butterflies and exchanges;
//   k_stockham_small    one whole row per thread for single-codelet lengths,
//                       with the tile staged through shared memory so that
//                       both HBM directions use 16-byte coalesced accesses.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "codelets.cuh"
#include "gbfft.h"

namespace gbfft {

// Shared-memory slot of tile element i: one complex of padding per 2^PS
// complex (PS = 0: no padding) to spread strided exchanges across banks.
template <int PS>
__device__ __forceinline__ int spad(int i) {
    return PS ? i + (i >> PS) : i;
}

template <int T, int N, int PS>
constexpr int smem_elems() {
    return PS ? (T * N - 1) + ((T * N - 1) >> PS) + 1 : T * N;
}

template <int A, int... Rest>
struct First {
    static constexpr int value = A;
};

// Total size of the concatenated stage twiddle blocks of a schedule.
template <int L, int... Rs>
struct StageTwiddles;
template <int L>
struct StageTwiddles<L> {
    static constexpr int value = 0;
};
template <int L, int R, int... Rest>
struct StageTwiddles<L, R, Rest...> {
    static constexpr int value = (L > 1 ? (R - 1) * L : 0) + StageTwiddles<L * R, Rest...>::value;
};

// Row addressing of a tile: element n of tile row t, complex type C (float2
// or double2).  ContigIO: rows are consecutive (row t at base + t*N).
template <int N, class C = float2>
struct ContigIO {
    const C* in;
    C* out;
    __device__ __forceinline__ C ld(int t, int n) const { return in[t * N + n]; }
    __device__ __forceinline__ void st(int t, int n, C v) const { out[t * N + n] = v; }
};
// An IO whose stores land in the same shared memory the last stage reads
// declares `static constexpr bool kSyncBeforeStore = true`: the stage engine
// then synchronises between the last stage's reads and its stores.
template <class IO, class = void>
struct SyncBeforeStore : std::false_type {};
template <class IO>
struct SyncBeforeStore<IO, std::void_t<decltype(IO::kSyncBeforeStore)>> : std::bool_constant<IO::kSyncBeforeStore> {};

// IndexedIO: row t starts at complex element off[t] of both buffers.
template <int N, class C = float2>
struct IndexedIO {
    const C* in;
    C* out;
    const long long* off;
    __device__ __forceinline__ C ld(int t, int n) const { return in[off[t] + n]; }
    __device__ __forceinline__ void st(int t, int n, C v) const { out[off[t] + n] = v; }
};

// Stage twiddles w^q, q = 1..15, of a radix-16 butterfly with index k from
// its stage block W[(q-1)*L + k]: the entries for q = 1, 2, 4, 8 are read, the
// other powers formed as products of those (at most three multiplications
// deep, each product of table values that are themselves correctly rounded).
template <class C>
__device__ __forceinline__ void twiddle_powers16(const C* __restrict__ blk, int L, int k, C (&w)[16]) {
    const C w1 = __ldg(&blk[k]), w2 = __ldg(&blk[L + k]);
    const C w4 = __ldg(&blk[3 * L + k]), w8 = __ldg(&blk[7 * L + k]);
    w[1] = w1;
    w[2] = w2;
    w[3] = cmul(w1, w2);
    w[4] = w4;
    w[5] = cmul(w1, w4);
    w[6] = cmul(w2, w4);
    w[7] = cmul(w[3], w4);
    w[8] = w8;
#pragma unroll
    for (int q = 9; q < 16; ++q) w[q] = cmul(w[q - 8], w8);
}

// The same for a radix-8 butterfly: q = 1, 2, 4 read, q = 3, 5, 6, 7 by products.
template <class C>
__device__ __forceinline__ void twiddle_powers8(const C* __restrict__ blk, int L, int k, C (&w)[8]) {
    const C w1 = __ldg(&blk[k]), w2 = __ldg(&blk[L + k]), w4 = __ldg(&blk[3 * L + k]);
    w[1] = w1;
    w[2] = w2;
    w[3] = cmul(w1, w2);
    w[4] = w4;
    w[5] = cmul(w1, w4);
    w[6] = cmul(w2, w4);
    w[7] = cmul(w[3], w4);
}

// Butterflies of radix R per thread when TPB threads share the T*N/R
// butterflies of a stage (the last round may leave threads idle).
template <int N, int T, int TPB, int R>
constexpr int stage_nb() {
    return (T * N / R + TPB - 1) / TPB;
}

// Stage-1 operands of this thread's butterflies, straight from HBM.
template <int N, int E, int T, int R, class IO, int TPB = T * N / E, class C>
__device__ __forceinline__ void gather_global(C (&v)[E], const IO& io, int nvalid) {
    constexpr int NB = stage_nb<N, T, TPB, R>(), NR = N / R, NBT = T * N / R;
    static_assert(NB * R <= E, "register capacity too small for this stage");
    const int tid = threadIdx.x;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int B = tid + u * TPB;
        if (NBT % TPB != 0 && B >= NBT) break;
        const int t = B / NR, j = B % NR;
#pragma unroll
        for (int q = 0; q < R; ++q) v[u * R + q] = (t < nvalid) ? io.ld(t, j + q * NR) : C{};
    }
}

// Stage operands from the shared-memory tile.
template <int N, int E, int T, int PS, int R, int TPB = T * N / E, class C>
__device__ __forceinline__ void gather_smem(C (&v)[E], const C* sm) {
    constexpr int NB = stage_nb<N, T, TPB, R>(), NR = N / R, NBT = T * N / R;
    static_assert(NB * R <= E, "register capacity too small for this stage");
    const int tid = threadIdx.x;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int B = tid + u * TPB;
        if (NBT % TPB != 0 && B >= NBT) break;
        const int t = B / NR, j = B % NR;
#pragma unroll
        for (int q = 0; q < R; ++q) v[u * R + q] = sm[spad<PS>(t * N + j + q * NR)];
    }
}

// Stages from the one whose operands `v` already holds to the end.  SYNC0:
// synchronise before the first shared-memory write (needed when earlier
// readers of the tile buffer may still be running).
// The stage loop with an explicit thread count TPB: stage s runs
// ceil(T*N/R_s / TPB) butterflies per thread (guarded when uneven), so a
// schedule may mix radices whose butterfly counts do not divide the threads.
template <int N, int S, int E, int T, int PS, int TPB, bool SYNC0, int TWO, int L, int R, int... Rest, class IO,
          class C>
__device__ __forceinline__ void run_stages_t(C (&v)[E], const IO& io, C* sm, const C* __restrict__ tw,
                                             int nvalid) {
    constexpr int NB = stage_nb<N, T, TPB, R>();  // butterflies per thread in this stage
    constexpr int NR = N / R;                     // butterflies per row
    constexpr int NBT = T * N / R;                // butterflies in the tile
    constexpr bool EVEN = NBT % TPB == 0;
    constexpr bool LAST = sizeof...(Rest) == 0;
    static_assert(NB * R <= E, "register capacity too small for this stage");
    const int tid = threadIdx.x;

#pragma unroll
    for (int u = 0; u < NB; ++u) {
        if (!EVEN && tid + u * TPB >= NBT) break;
        if constexpr (L > 1) {
            const int B = tid + u * TPB;
            const int k = (B % NR) % L;
            if constexpr (R == 16 && sizeof(C) == sizeof(float2)) {
                // FP32: 4 table reads per butterfly instead of 15 takes the twiddle loads off the
                // critical path of the large sizes (N = 2048: 96 -> 99.7 %, N = 4096: 95 -> 98.5 % of
                // the copy rate).  The FP64 path keeps the table reads: it is bound by the FP64 pipe,
                // where the products would cost more.
                C w[16];
                twiddle_powers16(tw + TWO, L, k, w);
#pragma unroll
                for (int q = 1; q < R; ++q) v[u * R + q] = twiddle<S>(v[u * R + q], w[q]);
            } else if constexpr (R == 8 && sizeof(C) == sizeof(float2)) {
                C w[8];
                twiddle_powers8(tw + TWO, L, k, w);
#pragma unroll
                for (int q = 1; q < R; ++q) v[u * R + q] = twiddle<S>(v[u * R + q], w[q]);
            } else {
#pragma unroll
                for (int q = 1; q < R; ++q)
                    v[u * R + q] = twiddle<S>(v[u * R + q], __ldg(&tw[TWO + (q - 1) * L + k]));
            }
        }
        Dft<S, R>::run(&v[u * R]);
    }
    if constexpr (LAST) {
        static_assert(L * R == N, "schedule must multiply to N");
        if constexpr (SyncBeforeStore<IO>::value) __syncthreads();
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = tid + u * TPB;
            if (!EVEN && B >= NBT) break;
            const int t = B / NR, j = B % NR;
            if (t < nvalid) {
#pragma unroll
                for (int q = 0; q < R; ++q) io.st(t, q * L + j, v[u * R + q]);
            }
        }
    } else {
        if constexpr (SYNC0) __syncthreads();
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = tid + u * TPB;
            if (!EVEN && B >= NBT) break;
            const int t = B / NR, j = B % NR;
            const int b = j / L, k = j % L;
#pragma unroll
            for (int q = 0; q < R; ++q) sm[spad<PS>(t * N + b * L * R + q * L + k)] = v[u * R + q];
        }
        __syncthreads();
        gather_smem<N, E, T, PS, First<Rest...>::value, TPB>(v, sm);
        run_stages_t<N, S, E, T, PS, TPB, true, TWO + (L > 1 ? (R - 1) * L : 0), L * R, Rest...>(v, io, sm, tw,
                                                                                                 nvalid);
    }
}

// Stages with TPB = T*N/E threads (every stage's butterflies divide evenly).
template <int N, int S, int E, int T, int PS, bool SYNC0, int TWO, int L, int R, int... Rest, class IO, class C>
__device__ __forceinline__ void run_stages(C (&v)[E], const IO& io, C* sm, const C* __restrict__ tw, int nvalid) {
    run_stages_t<N, S, E, T, PS, T * N / E, SYNC0, TWO, L, R, Rest...>(v, io, sm, tw, nvalid);
}

__device__ __forceinline__ int tile_rows(long long tile, int T, long long batch) {
    const long long rem = batch - tile * T;
    return rem < T ? (int)rem : T;
}

// Batched contiguous rows: row i of `in`/`out` starts at complex element i*N.
// One CTA per T rows; the last CTA may hold fewer (ragged tail).
template <int N, int S, int E, int T, int PS, int... Rs>
__global__ void __launch_bounds__(T * N / E) k_stockham_rows(const float2* in, float2* out,
                                                              const float2* __restrict__ tw, long long batch) {
    extern __shared__ float2 sm[];
    const long long tile = blockIdx.x;
    const int nvalid = tile_rows(tile, T, batch);
    float2 v[E];
    const ContigIO<N> io{in + tile * T * N, out + tile * T * N};
    gather_global<N, E, T, First<Rs...>::value>(v, io, nvalid);
    run_stages<N, S, E, T, PS, false, 0, 1, Rs...>(v, io, sm, tw, nvalid);
}

// Register capacity for a schedule run by TPB threads: the largest
// butterflies-per-thread times radix over its stages.
template <int N, int T, int TPB, int R, int... Rest>
constexpr int capacity_of_r() {
    constexpr int here = stage_nb<N, T, TPB, R>() * R;
    if constexpr (sizeof...(Rest) == 0) {
        return here;
    } else {
        constexpr int rest = capacity_of_r<N, T, TPB, Rest...>();
        return here > rest ? here : rest;
    }
}

// Contiguous rows with an explicit thread count (mixed-radix schedules).
template <int N, int S, int TPB, int T, int PS, int... Rs>
__global__ void __launch_bounds__(TPB) k_stockham_rows_t(const float2* in, float2* out,
                                                          const float2* __restrict__ tw, long long batch) {
    constexpr int E = capacity_of_r<N, T, TPB, Rs...>();
    extern __shared__ float2 sm[];
    const long long tile = blockIdx.x;
    const int nvalid = tile_rows(tile, T, batch);
    float2 v[E];
    const ContigIO<N> io{in + tile * T * N, out + tile * T * N};
    gather_global<N, E, T, First<Rs...>::value, ContigIO<N>, TPB>(v, io, nvalid);
    run_stages_t<N, S, E, T, PS, TPB, false, 0, 1, Rs...>(v, io, sm, tw, nvalid);
}

// The same on complex128 rows (FP64 arithmetic, double2 stage twiddles).
template <int N, int S, int TPB, int T, int PS, int... Rs>
__global__ void __launch_bounds__(TPB) k_stockham_rows_d(const double2* in, double2* out,
                                                          const double2* __restrict__ tw, long long batch) {
    constexpr int E = capacity_of_r<N, T, TPB, Rs...>();
    extern __shared__ double2 smd[];
    const long long tile = blockIdx.x;
    const int nvalid = tile_rows(tile, T, batch);
    double2 v[E];
    const ContigIO<N, double2> io{in + tile * T * N, out + tile * T * N};
    gather_global<N, E, T, First<Rs...>::value, ContigIO<N, double2>, TPB>(v, io, nvalid);
    run_stages_t<N, S, E, T, PS, TPB, false, 0, 1, Rs...>(v, io, smd, tw, nvalid);
}

// Persistent form with register prefetch of the next tile's stage-1 operands.
// In place is safe: a CTA reads tile i + gridDim.x before it writes tile i,
// and only this CTA ever writes tile i + gridDim.x.
template <int N, int S, int E, int T, int PS, int... Rs>
__global__ void __launch_bounds__(T * N / E) k_stockham_rows_pf(const float2* in, float2* out,
                                                                 const float2* __restrict__ tw, long long batch) {
    extern __shared__ float2 sm[];
    constexpr int R1 = First<Rs...>::value;
    const long long ntiles = (batch + T - 1) / T;
    long long tile = blockIdx.x;
    float2 nxt[E];
    if (tile < ntiles)
        gather_global<N, E, T, R1>(nxt, ContigIO<N>{in + tile * T * N, nullptr}, tile_rows(tile, T, batch));
    for (; tile < ntiles; tile += gridDim.x) {
        float2 v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = nxt[e];
        const long long next = tile + gridDim.x;
        if (next < ntiles)
            gather_global<N, E, T, R1>(nxt, ContigIO<N>{in + next * T * N, nullptr}, tile_rows(next, T, batch));
        run_stages<N, S, E, T, PS, true, 0, 1, Rs...>(v, ContigIO<N>{nullptr, out + tile * T * N}, sm, tw,
                                                      tile_rows(tile, T, batch));
    }
}

// ---------------------------------------------------------------------------
// Persistent kernel with TMA prefetch.  Each CTA walks tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; while it transforms tile i from a shared-memory
// staging buffer, the TMA engine already copies tile i + gridDim.x (one
// contiguous block of T rows) into the other staging buffer with a 1-D bulk
// copy (cp.async.bulk) that completes on an mbarrier.  Stage 1 then reads the
// staged tile, the stages exchange through the padded buffer as usual, and the
// last stage writes HBM directly.  Every wait on an mbarrier is bounded (a
// globaltimer deadline); on expiry the kernel records GBFFT_ERR_TIMEOUT in the
// status word, waits (bounded again) for its copies in flight and returns.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long gbfft_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for phase `parity` of an mbarrier; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
    const uint32_t addr = smem_u32(bar);
    const unsigned long long t0 = gbfft_globaltimer();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n"
            "}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (gbfft_globaltimer() - t0 > limit_ns) return false;
    }
}

// 1-D bulk copy global -> shared (16-byte aligned, size a multiple of 16),
// completing `bytes` of transaction count on `bar`.
__device__ __forceinline__ void tma_load_1d(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

constexpr unsigned long long kTmaWaitNs = 1000000000ull;  // 1 s bound on any copy wait

template <int N, int T, int PS>
constexpr int tma_smem_bytes() {
    return 2 * T * N * (int)sizeof(float2) + smem_elems<T, N, PS>() * (int)sizeof(float2) + 16;
}

template <int N, int S, int TPB, int T, int PS, int... Rs>
__global__ void __launch_bounds__(TPB) k_stockham_rows_tma(const float2* in, float2* out,
                                                            const float2* __restrict__ tw, long long batch,
                                                            int* status) {
    constexpr int E = capacity_of_r<N, T, TPB, Rs...>();
    extern __shared__ __align__(128) float2 smem_all[];
    float2* const stage0 = smem_all;
    float2* const stage1 = smem_all + T * N;
    float2* xbuf = smem_all + 2 * T * N;
    uint64_t* bars = reinterpret_cast<uint64_t*>(xbuf + smem_elems<T, N, PS>());
    const long long ntiles = (batch + T - 1) / T;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    long long tile = blockIdx.x;
    if (tid == 0 && tile < ntiles) {
        const uint32_t bytes = (uint32_t)(tile_rows(tile, T, batch) * N * sizeof(float2));
        mbar_expect_tx(&bars[0], bytes);
        tma_load_1d(stage0, in + tile * T * N, bytes, &bars[0]);
    }
    uint32_t phase0 = 0u, phase1 = 0u;
    for (int i = 0; tile < ntiles; tile += gridDim.x, ++i) {
        const int b = i & 1;
        float2* const cur = b ? stage1 : stage0;
        float2* const other = b ? stage0 : stage1;
        __syncthreads();  // the other staging buffer and the exchange buffer are free again
        const long long next = tile + gridDim.x;
        if (tid == 0 && next < ntiles) {
            const uint32_t bytes = (uint32_t)(tile_rows(next, T, batch) * N * sizeof(float2));
            fence_proxy_async_smem();
            mbar_expect_tx(&bars[b ^ 1], bytes);
            tma_load_1d(other, in + next * T * N, bytes, &bars[b ^ 1]);
        }
        const uint32_t par = b ? phase1 : phase0;
        const int ok = __syncthreads_and(mbar_wait(&bars[b], par, kTmaWaitNs) ? 1 : 0);
        if (!ok) {  // uniform decision: every thread leaves together
            if (tid == 0) atomicCAS(status, 0, (int)GBFFT_ERR_TIMEOUT);
            if (next < ntiles) mbar_wait(&bars[b ^ 1], b ? phase0 : phase1, kTmaWaitNs);
            return;
        }
        if (b) phase1 ^= 1u;
        else phase0 ^= 1u;
        const int nvalid = tile_rows(tile, T, batch);
        float2 v[E];
        gather_global<N, E, T, First<Rs...>::value, ContigIO<N>, TPB>(v, ContigIO<N>{cur, nullptr}, nvalid);
        run_stages_t<N, S, E, T, PS, TPB, true, 0, 1, Rs...>(v, ContigIO<N>{nullptr, out + tile * T * N}, xbuf, tw,
                                                            nvalid);
    }
}

// One row per thread (T rows per CTA) for a length with a single codelet.
// The tile is copied HBM -> shared memory with 16-byte coalesced loads, each
// thread transforms its row in registers, and the tile goes back with 16-byte
// coalesced stores.  Row pitch N + 2 complex keeps the per-thread row accesses
// conflict-free and the 16-byte slots aligned.  Requires even N.
template <int N, int S, int T>
__global__ void __launch_bounds__(T) k_stockham_small(const float2* in, float2* out, const float2* __restrict__ tw,
                                                       long long batch) {
    static_assert(N % 2 == 0, "staged rows need an even length");
    constexpr int P = N + 2;
    extern __shared__ float2 sm[];
    const long long tile = blockIdx.x;
    const int nvalid = tile_rows(tile, T, batch);
    const int tid = threadIdx.x;
    const float4* g4 = reinterpret_cast<const float4*>(in + tile * T * N);
    float4* o4 = reinterpret_cast<float4*>(out + tile * T * N);
    const int nf = nvalid * (N / 2);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const int f = tid + i * T;
        if (f < nf) {
            const int row = (2 * f) / N, col = (2 * f) % N;
            *reinterpret_cast<float4*>(&sm[row * P + col]) = g4[f];
        }
    }
    __syncthreads();
    float2 v[N];
#pragma unroll
    for (int n = 0; n < N; n += 2) {
        const float4 p = *reinterpret_cast<const float4*>(&sm[tid * P + n]);
        v[n] = make_float2(p.x, p.y);
        v[n + 1] = make_float2(p.z, p.w);
    }
    Dft<S, N>::run(v);
#pragma unroll
    for (int n = 0; n < N; n += 2)
        *reinterpret_cast<float4*>(&sm[tid * P + n]) = make_float4(v[n].x, v[n].y, v[n + 1].x, v[n + 1].y);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const int f = tid + i * T;
        if (f < nf) {
            const int row = (2 * f) / N, col = (2 * f) % N;
            o4[f] = *reinterpret_cast<const float4*>(&sm[row * P + col]);
        }
    }
}

// Row pitch (complex) of the staged tile: an odd number of 16-byte units per
// row, so that the 16-byte row accesses of a warp spread over all banks
// (N + 2 when that is odd in 16-byte units, else N + 4: at N = 14 a pitch of
// 16 complex put every row on the same banks and ran at half the rate).
constexpr int small2_pitch(int n) { return ((n + 2) / 2) % 2 == 1 ? n + 2 : n + 4; }

// One row per thread for a length N = R1 * R2 (a mixed-radix length too long
// for one codelet, N <= 56): the tile is staged through shared memory as in
// k_stockham_small, and each thread runs both Stockham stages of its row in
// registers.  Stage 1 (radix R1, L = 1): butterfly b < R2 takes x[b + q*R2]
// and writes y[b*R1 + q]; stage 2 (radix R2, L = R1): butterfly k < R1 takes
// y[k + q*R1] * w_N^(q*k) from the plan's stage block W[(q-1)*R1 + k] and
// writes the output element q*R1 + k (natural order).
template <int N, int S, int T, int R1, int R2>
__global__ void __launch_bounds__(T) k_stockham_small2(const float2* in, float2* out, const float2* __restrict__ tw,
                                                        long long batch) {
    static_assert(N == R1 * R2 && N % 2 == 0, "staged rows need an even length R1 * R2");
    constexpr int P = small2_pitch(N);
    extern __shared__ float2 sm[];
    const long long tile = blockIdx.x;
    const int nvalid = tile_rows(tile, T, batch);
    const int tid = threadIdx.x;
    const float4* g4 = reinterpret_cast<const float4*>(in + tile * T * N);
    float4* o4 = reinterpret_cast<float4*>(out + tile * T * N);
    const int nf = nvalid * (N / 2);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const int f = tid + i * T;
        if (f < nf) {
            const int row = (2 * f) / N, col = (2 * f) % N;
            *reinterpret_cast<float4*>(&sm[row * P + col]) = g4[f];
        }
    }
    __syncthreads();
    float2 v[N];
#pragma unroll
    for (int n = 0; n < N; n += 2) {
        const float4 p = *reinterpret_cast<const float4*>(&sm[tid * P + n]);
        v[n] = make_float2(p.x, p.y);
        v[n + 1] = make_float2(p.z, p.w);
    }
    float2 y[N];
#pragma unroll
    for (int b = 0; b < R2; ++b) {
        float2 a[R1];
#pragma unroll
        for (int q = 0; q < R1; ++q) a[q] = v[b + q * R2];
        Dft<S, R1>::run(a);
#pragma unroll
        for (int q = 0; q < R1; ++q) y[b * R1 + q] = a[q];
    }
#pragma unroll
    for (int k = 0; k < R1; ++k) {
        float2 a[R2];
        a[0] = y[k];
#pragma unroll
        for (int q = 1; q < R2; ++q) a[q] = k == 0 ? y[k + q * R1] : twiddle<S>(y[k + q * R1], __ldg(&tw[(q - 1) * R1 + k]));
        Dft<S, R2>::run(a);
#pragma unroll
        for (int q = 0; q < R2; ++q) v[q * R1 + k] = a[q];
    }
#pragma unroll
    for (int n = 0; n < N; n += 2)
        *reinterpret_cast<float4*>(&sm[tid * P + n]) = make_float4(v[n].x, v[n].y, v[n + 1].x, v[n + 1].y);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const int f = tid + i * T;
        if (f < nf) {
            const int row = (2 * f) / N, col = (2 * f) % N;
            o4[f] = *reinterpret_cast<const float4*>(&sm[row * P + col]);
        }
    }
}

}  // namespace gbfft
