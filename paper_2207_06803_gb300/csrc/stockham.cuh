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
// HBM (again consecutive threads, consecutive elements).  Twiddles come from a
// per-plan table tw[e] = exp(-2*pi*i*e/N) (FP64-generated, stored as float2);
// w_{L'}^(q*k) is tw[q*k*(N/L')], and the inverse uses the conjugate.
#pragma once
#include <cuda_runtime.h>

#include "codelets.cuh"

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

template <int N, int S, int E, int T, int PS, int L, bool FIRST, int R, int... Rest>
__device__ __forceinline__ void stages_rows(float2 (&v)[E], const float2* gin, float2* gout, float2* sm,
                                            const float2* __restrict__ tw, int nvalid) {
    constexpr int TPB = T * N / E;
    constexpr int NB = E / R;  // butterflies per thread in this stage
    constexpr int NR = N / R;  // butterflies per row
    constexpr bool LAST = sizeof...(Rest) == 0;
    static_assert(E % R == 0, "radix must divide the elements held per thread");
    const int tid = threadIdx.x;

#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int B = tid + u * TPB;
        const int t = B / NR, j = B % NR;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int n = j + q * NR;
            if constexpr (FIRST) {
                v[u * R + q] = (t < nvalid) ? gin[t * N + n] : make_float2(0.f, 0.f);
            } else {
                v[u * R + q] = sm[spad<PS>(t * N + n)];
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        if constexpr (L > 1) {
            const int B = tid + u * TPB;
            const int k = (B % NR) % L;
#pragma unroll
            for (int q = 1; q < R; ++q)
                v[u * R + q] = twiddle<S>(v[u * R + q], __ldg(&tw[q * k * (N / (L * R))]));
        }
        Dft<S, R>::run(&v[u * R]);
    }
    if constexpr (LAST) {
        static_assert(L * R == N, "schedule must multiply to N");
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = tid + u * TPB;
            const int t = B / NR, j = B % NR;
            if (t < nvalid) {
#pragma unroll
                for (int q = 0; q < R; ++q) gout[t * N + q * L + j] = v[u * R + q];
            }
        }
    } else {
        if constexpr (!FIRST) __syncthreads();  // all reads of the previous exchange are done
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = tid + u * TPB;
            const int t = B / NR, j = B % NR;
            const int b = j / L, k = j % L;
#pragma unroll
            for (int q = 0; q < R; ++q) sm[spad<PS>(t * N + b * L * R + q * L + k)] = v[u * R + q];
        }
        __syncthreads();
        stages_rows<N, S, E, T, PS, L * R, false, Rest...>(v, gin, gout, sm, tw, nvalid);
    }
}

// Batched contiguous rows: row i of `in`/`out` starts at complex element i*N.
// One CTA per T rows; the last CTA may hold fewer (ragged tail).
template <int N, int S, int E, int T, int PS, int... Rs>
__global__ void __launch_bounds__(T * N / E) k_stockham_rows(const float2* in, float2* out,
                                                              const float2* __restrict__ tw, long long batch) {
    extern __shared__ float2 sm[];
    const long long r0 = (long long)blockIdx.x * T;
    const long long rem = batch - r0;
    const int nvalid = rem < T ? (int)rem : T;
    float2 v[E];
    stages_rows<N, S, E, T, PS, 1, true, Rs...>(v, in + r0 * N, out + r0 * N, sm, tw, nvalid);
}

}  // namespace gbfft
