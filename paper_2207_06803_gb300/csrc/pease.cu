// Pease's constant-geometry factorisation of DFT_N, N = R^t (one of the other
// factorisation schemes the paper names beside Stockham, Sec. II), as a
// single-pass kernel variant.
//
// From Eq. 2 with K = R (DFT_N = (DFT_R ⊗ I_{N/R}) D^N_{N/R} (I_R ⊗ DFT_{N/R}) Pi^N_R)
// and Pi^N_R (A ⊗ I_R) = (I_R ⊗ A) Pi^N_R, unrolled over the t digits:
//     DFT_N = G_t ... G_1 Rev_N,
//     G_s   = (DFT_R ⊗ I_{N/R}) (D^{R^s}_{R^{s-1}} ⊗ I_{R^{t-s}}) Pi^N_R,
//     Rev_N = (I_R ⊗ Rev_{N/R}) Pi^N_R,  Rev_R = I_R    (base-R digit reversal).
// Every stage has the same geometry: butterfly j < N/R reads the R
// consecutive elements z[j R + q], multiplies them by w_{R^s}^(q k) with
// k = floor(j / R^(t-s)), and writes z'[p N/R + j] for p < R.  The first
// stage reads the digit-reversed input straight from HBM, z_0[j R + q] =
// x[q N/R + rev_{t-1}(j)]; the last stage's writes are the natural order.
// The stage twiddles w_{R^s}^(q k), k < R^(s-1), are the stage blocks of the
// all-R Stockham schedule (the same table, W[(q-1) L + k] with L = R^(s-1)).
// Between stages the tile is exchanged through padded shared memory.
//
// What differs from the Stockham kernels is only the data flow: stride-R
// contiguous reads and stride-N/R writes at every stage, and a gather of the
// first stage's operands in digit-reversed order, which is the cost the
// constant geometry brings on a GPU.  For rows up to N = 512 the gather
// reads HBM directly (scattered 8-byte loads whose sectors the rest of the
// tile uses while they are still in L1); at N = 4096 the tile is first copied
// into shared memory with coalesced 16-byte loads and the gather reads it
// from there (one more shared-memory pass than Stockham: 0.84 of Stockham's
// rate against 0.48 for the direct gather; at N = 512 the direct gather is
// the faster, 0.88 against 0.78).
#include <cuda_runtime.h>

#include "internal.h"
#include "stockham.cuh"

namespace gbfft {
namespace {

constexpr int ipow(int r, int e) { return e == 0 ? 1 : r * ipow(r, e - 1); }
constexpr int ilog(int n, int r) { return n == 1 ? 0 : 1 + ilog(n / r, r); }

// The M base-R digits of x in reverse order.
template <int R, int M>
__device__ __forceinline__ int digit_reverse(int x) {
    int y = 0;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        y = y * R + x % R;
        x /= R;
    }
    return y;
}

template <int N, int S, int R, int T, int TPB, int PS, int s>
__device__ __forceinline__ void pease_stages(float2 (&v)[(T * N / R / TPB) * R], float2* sm,
                                             const float2* __restrict__ tw, float2* y, int nvalid) {
    constexpr int TS = ilog(N, R);
    constexpr int NR = N / R, NB = T * NR / TPB;
    constexpr int L = ipow(R, s - 1);   // the stage's twiddle span, R^(s-1)
    constexpr int DIV = ipow(R, TS - s);  // k = floor(j / R^(t-s))
    const int tid = threadIdx.x;
    if constexpr (s > 1) {
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = tid + u * TPB;
            const int t = B / NR, j = B % NR;
#pragma unroll
            for (int q = 0; q < R; ++q) v[u * R + q] = sm[spad<PS>(t * N + j * R + q)];
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int j = (tid + u * TPB) % NR;
            const int k = j / DIV;
            const float2* blk = tw + (L - R);  // stage blocks of the all-R schedule: L - R before this one
            if constexpr (R == 16) {
                float2 w[16];
                twiddle_powers16(blk, L, k, w);
#pragma unroll
                for (int q = 1; q < R; ++q) v[u * R + q] = twiddle<S>(v[u * R + q], w[q]);
            } else if constexpr (R == 8) {
                float2 w[8];
                twiddle_powers8(blk, L, k, w);
#pragma unroll
                for (int q = 1; q < R; ++q) v[u * R + q] = twiddle<S>(v[u * R + q], w[q]);
            } else {
#pragma unroll
                for (int q = 1; q < R; ++q) v[u * R + q] = twiddle<S>(v[u * R + q], __ldg(&blk[(q - 1) * L + k]));
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) Dft<S, R>::run(&v[u * R]);
    if constexpr (s < TS) {
        if constexpr (s > 1) __syncthreads();  // every read of the tile precedes the first write
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = tid + u * TPB;
            const int t = B / NR, j = B % NR;
#pragma unroll
            for (int p = 0; p < R; ++p) sm[spad<PS>(t * N + p * NR + j)] = v[u * R + p];
        }
        __syncthreads();
        pease_stages<N, S, R, T, TPB, PS, s + 1>(v, sm, tw, y, nvalid);
    } else {
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = tid + u * TPB;
            const int t = B / NR, j = B % NR;
            if (t < nvalid) {
#pragma unroll
                for (int p = 0; p < R; ++p) y[t * N + p * NR + j] = v[u * R + p];
            }
        }
    }
}

// One tile of T rows per CTA; the last CTA may hold fewer (ragged tail).
template <int N, int S, int R, int T, int TPB, int PS>
__global__ void __launch_bounds__(TPB) k_pease_rows(const float2* in, float2* out, const float2* __restrict__ tw,
                                                     long long batch) {
    constexpr int TS = ilog(N, R);
    constexpr int NR = N / R, NB = T * NR / TPB;
    static_assert(ipow(R, TS) == N && TS >= 2, "Pease form: N a power of R with at least two stages");
    static_assert((T * NR) % TPB == 0, "the butterflies of a stage must divide evenly over the threads");
    extern __shared__ float2 sm[];
    const long long tile = blockIdx.x;
    const int nvalid = tile_rows(tile, T, batch);
    const float2* x = in + tile * T * N;
    const int tid = threadIdx.x;
    float2 v[NB * R];
    // z_0 = Rev_N x: the operands of butterfly j are x[q N/R + rev_{t-1}(j)]
    if constexpr (N <= 512) {
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = tid + u * TPB;
            const int t = B / NR, j = B % NR;
            const int jr = digit_reverse<R, TS - 1>(j);
#pragma unroll
            for (int q = 0; q < R; ++q)
                v[u * R + q] = (t < nvalid) ? __ldg(x + t * N + q * NR + jr) : make_float2(0.f, 0.f);
        }
    } else {
        static_assert((T * N) % (2 * TPB) == 0, "the tile copy takes two complex per thread per step");
        const float4* x4 = reinterpret_cast<const float4*>(x);
#pragma unroll 4
        for (int i = 2 * tid; i < T * N; i += 2 * TPB) {
            const float4 w = (i / N < nvalid) ? __ldg(x4 + i / 2) : make_float4(0.f, 0.f, 0.f, 0.f);
            sm[spad<PS>(i)] = make_float2(w.x, w.y);
            sm[spad<PS>(i + 1)] = make_float2(w.z, w.w);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int B = tid + u * TPB;
            const int t = B / NR, j = B % NR;
            const int jr = digit_reverse<R, TS - 1>(j);
#pragma unroll
            for (int q = 0; q < R; ++q) v[u * R + q] = sm[spad<PS>(t * N + q * NR + jr)];
        }
        __syncthreads();  // the gather precedes stage 1's writes into the tile
    }
    pease_stages<N, S, R, T, TPB, PS, 1>(v, sm, tw, out + tile * T * N, nvalid);
}

template <int N, int R, int T, int TPB, int PS>
RowsVariant make_pease_variant() {
    constexpr int TS = ilog(N, R);
    RowsVariant v{};
    v.kind = kRowsPease;
    v.n = N;
    v.e = (T * N / R / TPB) * R;
    v.rows = T;
    v.tpb = TPB;
    v.ps = PS;
    v.nstages = TS;
    for (int i = 0; i < TS; ++i) v.radix[i] = R;
    v.smem = smem_elems<T, N, PS>() * (int)sizeof(float2);
    v.kfwd = (const void*)&k_pease_rows<N, -1, R, T, TPB, PS>;
    v.kinv = (const void*)&k_pease_rows<N, +1, R, T, TPB, PS>;
    return v;
}

// Tile shapes as the Stockham variants of the same lengths: 256 threads, one
// butterfly (two at N = 512) per thread per stage.
const RowsVariant kPease[] = {
    make_pease_variant<64, 8, 32, 256, 3>(),
    make_pease_variant<256, 16, 16, 256, 4>(),
    make_pease_variant<512, 8, 8, 256, 4>(),
    make_pease_variant<4096, 16, 1, 256, 4>(),
};

}  // namespace

const RowsVariant* rows_variants_pease(int* count) {
    *count = (int)(sizeof(kPease) / sizeof(kPease[0]));
    return kPease;
}

}  // namespace gbfft
