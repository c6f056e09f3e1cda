// Column transforms: the two passes of Eq. 2 for long rows.
//
// For N = K * M, Eq. 2 reads DFT_N = (DFT_K (x) I_M) D^N_M (I_K (x) DFT_M) Pi^N_K.
// Viewing a row x as a K-column matrix (element m of column k at x[m*K + k]):
//
//   pass 1  z[k*M + j1] = w_N^(j1*k) * sum_m w_M^(j1*m) x[m*K + k]
//           Pi^N_K is the column gather, I_K (x) DFT_M the column transforms,
//           D^N_M the twiddle applied on the way out; z is the plan workspace.
//   pass 2  y[j2*M + j1] = sum_k w_K^(j2*k) z[k*M + j1]
//           DFT_K (x) I_M: length-K transforms down the M columns of z.
//
// Both passes are batches of strided transforms: a CTA takes C consecutive
// columns of one row's matrix, so that for every element index the C values
// are contiguous in HBM (C*8 = 64 or 128 bytes).  Within the CTA each column is
// transformed by the same Stockham stages as the row kernel, with the
// butterfly-to-thread map column-fastest (consecutive threads = consecutive
// columns).  Pass 1 writes its output through shared memory so that the
// workspace rows it produces (C whole rows of length M, contiguous) leave with
// consecutive threads on consecutive elements, multiplying by the D^N_M table
// P[k*M + j1] = w_N^(j1*k) (same layout as z, so those reads are contiguous).
#pragma once
#include <cuda_runtime.h>

#include "codelets.cuh"
#include "stockham.cuh"

namespace gbfft {

enum ColsMode : int { kColsPass1 = 1, kColsPass2 = 2 };

// Shared-memory slot of element (column c, index n): pitch C + 1 per index.
template <int C>
__device__ __forceinline__ int cslot(int c, int n) {
    return n * (C + 1) + c;
}

template <int LEN, int E, int C, int R>
__device__ __forceinline__ void cols_gather_global(float2 (&v)[E], const float2* gin, int ncols) {
    constexpr int TPB = C * LEN / E, NB = E / R, NR = LEN / R;
    const int tid = threadIdx.x;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int B = tid + u * TPB;
        const int c = B % C, j = B / C;
#pragma unroll
        for (int q = 0; q < R; ++q) v[u * R + q] = gin[(long long)(j + q * NR) * ncols + c];
    }
}

template <int LEN, int E, int C, int R>
__device__ __forceinline__ void cols_gather_smem(float2 (&v)[E], const float2* sm) {
    constexpr int TPB = C * LEN / E, NB = E / R, NR = LEN / R;
    const int tid = threadIdx.x;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int B = tid + u * TPB;
        const int c = B % C, j = B / C;
#pragma unroll
        for (int q = 0; q < R; ++q) v[u * R + q] = sm[cslot<C>(c, j + q * NR)];
    }
}

// Arguments shared by every stage of a column launch.
struct ColsArgs {
    float2* gout;                  // pass 2: this CTA's first output column; pass 1: its first z row
    const float2* __restrict__ tw; // stage twiddle blocks for length LEN
    const float2* __restrict__ post; // pass 1: D^N_M table slice of this CTA (C rows of M)
    int ncols;                     // columns of the matrix (= its row stride in elements)
};

template <int LEN, int S, int E, int C, int MODE, bool SYNC0, int TWO, int L, int R, int... Rest>
__device__ __forceinline__ void cols_run_stages(float2 (&v)[E], float2* sm, const ColsArgs& a) {
    constexpr int TPB = C * LEN / E;
    constexpr int NB = E / R;
    constexpr int NR = LEN / R;
    constexpr bool LAST = sizeof...(Rest) == 0;
    static_assert(E % R == 0, "radix must divide the elements held per thread");
    const int tid = threadIdx.x;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        if constexpr (L > 1) {
            const int B = tid + u * TPB;
            const int k = (B / C) % L;
#pragma unroll
            for (int q = 1; q < R; ++q) v[u * R + q] = twiddle<S>(v[u * R + q], __ldg(&a.tw[TWO + (q - 1) * L + k]));
        }
        Dft<S, R>::run(&v[u * R]);
    }
    if constexpr (LAST) {
        static_assert(L * R == LEN, "schedule must multiply to the column length");
        if constexpr (MODE == kColsPass2) {
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                const int B = tid + u * TPB;
                const int c = B % C, j = B / C;
#pragma unroll
                for (int q = 0; q < R; ++q) a.gout[(long long)(q * L + j) * a.ncols + c] = v[u * R + q];
            }
        } else {
            if constexpr (SYNC0) __syncthreads();
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                const int B = tid + u * TPB;
                const int c = B % C, j = B / C;
#pragma unroll
                for (int q = 0; q < R; ++q) sm[cslot<C>(c, q * L + j)] = v[u * R + q];
            }
            __syncthreads();
            // C consecutive z rows of length LEN: element (c, n) at c*LEN + n.
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int idx = tid + i * TPB;
                const int c = idx / LEN, n = idx % LEN;
                a.gout[idx] = twiddle<S>(sm[cslot<C>(c, n)], __ldg(&a.post[idx]));
            }
        }
    } else {
        if constexpr (SYNC0) __syncthreads();
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = tid + u * TPB;
            const int c = B % C, j = B / C;
            const int b = j / L, k = j % L;
#pragma unroll
            for (int q = 0; q < R; ++q) sm[cslot<C>(c, b * L * R + q * L + k)] = v[u * R + q];
        }
        __syncthreads();
        cols_gather_smem<LEN, E, C, First<Rest...>::value>(v, sm);
        cols_run_stages<LEN, S, E, C, MODE, true, TWO + (L > 1 ? (R - 1) * L : 0), L * R, Rest...>(v, sm, a);
    }
}

// One CTA = C consecutive columns of one batch row's LEN x ncols matrix
// (row length n_total = LEN * ncols).  Pass 1: `out` is the workspace z and
// `post` the D^N_M table; pass 2: `out` is y and `post` is unused.
template <int LEN, int S, int E, int C, int MODE, int... Rs>
__global__ void __launch_bounds__(C * LEN / E) k_stockham_cols(const float2* in, float2* out,
                                                                const float2* __restrict__ tw,
                                                                const float2* __restrict__ post, int ncols) {
    extern __shared__ float2 sm[];
    const int groups = ncols / C;
    const long long b = blockIdx.x / groups;
    const int g = blockIdx.x % groups;
    const long long n_total = (long long)LEN * ncols;
    const float2* gin = in + b * n_total + (long long)g * C;
    ColsArgs a;
    a.tw = tw;
    a.ncols = ncols;
    if constexpr (MODE == kColsPass1) {
        a.gout = out + b * n_total + (long long)g * C * LEN;
        a.post = post + (long long)g * C * LEN;
    } else {
        a.gout = out + b * n_total + (long long)g * C;
        a.post = nullptr;
    }
    float2 v[E];
    cols_gather_global<LEN, E, C, First<Rs...>::value>(v, gin, ncols);
    cols_run_stages<LEN, S, E, C, MODE, false, 0, 1, Rs...>(v, sm, a);
}

}  // namespace gbfft
