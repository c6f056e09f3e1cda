// One-pass transforms for 4096 < N <= 32768 on thread-block clusters.
//
// Eq. 2 with N = K * M, DFT_N = (DFT_K (x) I_M) D^N_M (I_K (x) DFT_M) Pi^N_K,
// run by a cluster of K CTAs (K = 2, 4, 8) on one row, the row staying on chip
// between the factors: CTA k owns column k of the K x M view.
//   A. CTA k reads the contiguous block [k*M, (k+1)*M) of the row from HBM and
//      sends element i to column i mod K, slot i div K (Pi^N_K) in the
//      distributed shared memory of the cluster.
//   B. Each CTA transforms its column with the single-pass Stockham engine
//      (I_K (x) DFT_M: the column's schedule, exchanges in its own shared
//      memory) and multiplies by its slice of D^N_M, w_N^(j1*k).
//   C. CTA c takes outputs j1 in [c*M/K, (c+1)*M/K): it reads z_k[j1] from all
//      K columns, applies DFT_K (DFT_K (x) I_M) and writes y[j2*M + j1] to HBM,
//      consecutive threads on consecutive j1.
// One HBM round trip instead of the two of the two-pass form; the exchanges
// between the factors go through distributed shared memory.  The cluster
// barriers are hardware barriers of the co-scheduled cluster (no spin on
// memory), every CTA of a cluster runs the same sequence of them, the first
// precedes any access to another CTA's shared memory (which is valid only once
// that CTA runs) and the last follows every such access (so that no CTA exits
// while its shared memory is still read).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "stockham.cuh"

namespace cg = cooperative_groups;

namespace gbfft {
namespace {

// A cluster barrier that orders no memory: arrive.relaxed lets a CTA pass
// without first waiting for its outstanding global loads and stores, which
// the release fence of cluster.sync() would.  Used where the barrier only
// has to establish that every CTA has started, or that every CTA is done
// reading the others' shared memory (its remote loads have returned: the
// values were consumed before the arrive in program order).
__device__ __forceinline__ void cluster_sync_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory");
}

// The column's I/O for the Stockham engine: it reads the column from shared
// memory and writes it back multiplied by the column's slice of D^N_M.  The
// column lives in the stages' own (padded) exchange buffer, so the engine
// synchronises before the first exchange (SYNC0) and before these stores.
template <int S, int PS>
struct ColumnIO {
    static constexpr bool kSyncBeforeStore = true;
    const float2* in;
    float2* out;
    const float2* __restrict__ post;  // w_N^(j1*k), j1 < M, of this CTA's column k
    __device__ __forceinline__ float2 ld(int, int n) const { return in[spad<PS>(n)]; }
    __device__ __forceinline__ void st(int, int n, float2 v) const {
        out[spad<PS>(n)] = twiddle<S>(v, __ldg(post + n));
    }
};

// VA: phase A by groups of K consecutive elements (16-byte loads; each destination column receives
// consecutive slots from consecutive threads), else element by element (8-byte loads at stride TPB).
template <int N, int K, int S, int TPB, int PS, bool VA, int MINB, int... Rs>
__global__ void __cluster_dims__(K, 1, 1) __launch_bounds__(TPB, MINB)
    k_stockham_cluster(const float2* in, float2* out, const float2* __restrict__ tw, long long batch) {
    constexpr int M = N / K;
    constexpr int E = capacity_of_r<M, 1, TPB, Rs...>();
    constexpr int STW = StageTwiddles<1, Rs...>::value;  // the column schedule's stage blocks; D^N_M follows
    static_assert((Rs * ...) == M, "column schedule must multiply to N / K");
    static_assert(M % TPB == 0 && M % K == 0, "column and output slices must split evenly");
    extern __shared__ float2 csm[];
    float2* const col = csm;  // column k, later z_k (padded slots); also the stages' exchange buffer
    cg::cluster_group cluster = cg::this_cluster();
    const int k = (int)cluster.block_rank();
    const long long row = blockIdx.x / K;  // one row per cluster; the grid holds exactly batch clusters
    const int tid = threadIdx.x;
    (void)batch;

    // A. block k of the row -> columns (Pi^N_K); all loads are issued before the remote stores.
    // Element k*M + i goes to column (k*M + i) mod K, slot (k*M + i) div K.  Another CTA's shared
    // memory may be written only once that CTA is running: the cluster barrier below is passed
    // only when every CTA of the cluster has started.
    const float2* x = in + row * N + (long long)k * M;
    if constexpr (VA) {
        // thread g takes the K consecutive elements g*K + q: element q goes to column q, slot
        // k*M/K + g, so for each q consecutive threads write consecutive slots of one column
        constexpr int JG = M / K;     // groups of K elements in the block
        constexpr int NG = JG / TPB;  // groups per thread
        static_assert(JG % TPB == 0 && K % 2 == 0, "the block splits into whole groups per thread");
        const float4* x4 = reinterpret_cast<const float4*>(x);
        float2 a[NG][K];
#pragma unroll
        for (int e = 0; e < NG; ++e) {
            const int g = tid + e * TPB;
#pragma unroll
            for (int h = 0; h < K / 2; ++h) {
                const float4 w = x4[g * (K / 2) + h];
                a[e][2 * h] = make_float2(w.x, w.y);
                a[e][2 * h + 1] = make_float2(w.z, w.w);
            }
        }
        cluster_sync_relaxed();  // every CTA of the cluster runs: its shared memory may be written
        const int base = spad<PS>(k * JG + tid);
#pragma unroll
        for (int q = 0; q < K; ++q) {
            float2* d = cluster.map_shared_rank(col + base, q);
#pragma unroll
            for (int e = 0; e < NG; ++e) d[spad<PS>(k * JG + tid + e * TPB) - base] = a[e][q];
        }
    } else {
        constexpr int NE = M / TPB;
        float2 a[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) a[e] = x[tid + e * TPB];
        cluster_sync_relaxed();  // every CTA of the cluster runs: its shared memory may be written
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int i = k * M + tid + e * TPB;
            float2* dst = cluster.map_shared_rank(col, i % K);
            dst[spad<PS>(i / K)] = a[e];
        }
    }
    cluster.sync();

    // B. I_K (x) DFT_M on this column, then D^N_M
    const ColumnIO<S, PS> io{col, col, tw + STW + (long long)k * M};
    float2 v[E];
    gather_global<M, E, 1, First<Rs...>::value, ColumnIO<S, PS>, TPB>(v, io, 1);
    run_stages_t<M, S, E, 1, PS, TPB, true, 0, 1, Rs...>(v, io, col, tw, 1);
    cluster.sync();

    // C. DFT_K (x) I_M across the columns, straight to HBM
    constexpr int J = M / K;
    float2* y = out + row * N;
    const float2* cols[K];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) cols[kk] = cluster.map_shared_rank(col, kk);
    constexpr int NJ = (J + TPB - 1) / TPB;  // outputs per thread: every remote load issued first
    float2 a[NJ][K];
#pragma unroll
    for (int e = 0; e < NJ; ++e) {
        const int jj = tid + e * TPB;
        if (jj < J) {
#pragma unroll
            for (int kk = 0; kk < K; ++kk) a[e][kk] = cols[kk][spad<PS>(k * J + jj)];
        }
    }
#pragma unroll
    for (int e = 0; e < NJ; ++e) {
        const int jj = tid + e * TPB;
        if (jj < J) {
            const int j1 = k * J + jj;
            Dft<S, K>::run(a[e]);
#pragma unroll
            for (int j2 = 0; j2 < K; ++j2) y[(long long)j2 * M + j1] = a[e][j2];
        }
    }
    cluster_sync_relaxed();  // no CTA leaves while the others still read its column
}

template <int N, int K, int TPB, int PS, bool VA, int MINB, int... Rs>
RowsVariant make_cluster_variant() {
    constexpr int M = N / K;
    return RowsVariant{kRowsCluster,
                       N,
                       capacity_of_r<M, 1, TPB, Rs...>(),
                       1,
                       TPB,
                       PS,
                       (int)sizeof...(Rs) + 1,
                       {Rs..., K},
                       (int)(smem_elems<1, M, PS>() * sizeof(float2)),
                       (const void*)&k_stockham_cluster<N, K, -1, TPB, PS, VA, MINB, Rs...>,
                       (const void*)&k_stockham_cluster<N, K, +1, TPB, PS, VA, MINB, Rs...>};
}

// Register caps from __launch_bounds__(TPB, 1024 / TPB): up to 16 complex per thread.
#define GBFFT_CLUSTER(N, K, TPB, PS, VA, ...) make_cluster_variant<N, K, TPB, PS, VA, 1024 / TPB, __VA_ARGS__>()
// Two CTAs per SM whatever TPB (up to 128 registers): schedules with up to 32 complex per thread.
#define GBFFT_CLUSTER2(N, K, TPB, PS, VA, ...) make_cluster_variant<N, K, TPB, PS, VA, 2, __VA_ARGS__>()

// The radix list of a variant is the column schedule followed by K.  The
// first entry of each length is its cluster default: a CTA pair whose column
// schedule opens with a composite p * 2^j stage (three stages: the
// single-pass schedules of those lengths) where the length has an odd factor;
// the radix-p-first schedules (four stages) and wider clusters follow as
// alternatives.  The grouped phase A (VA) measured faster everywhere but on
// N = 8192 and 16384 with K = 2, whose kernels spill with it (8192: 3.31
// against 3.57 TB/s).
const RowsVariant kCluster[] = {
    GBFFT_CLUSTER(5120, 2, 160, 0, true, 20, 8, 16),
    GBFFT_CLUSTER(5120, 2, 160, 5, true, 5, 16, 16, 2),
    GBFFT_CLUSTER(6144, 2, 192, 5, true, 24, 8, 16),
    GBFFT_CLUSTER(6144, 2, 192, 4, true, 3, 16, 16, 4),
    GBFFT_CLUSTER(7168, 2, 256, 0, true, 14, 16, 16),
    GBFFT_CLUSTER(7168, 2, 224, 4, true, 7, 16, 16, 2),
    GBFFT_CLUSTER(8192, 2, 256, 4, false, 16, 16, 16),
    GBFFT_CLUSTER(8192, 4, 128, 4, true, 16, 16, 8),
    GBFFT_CLUSTER(10240, 2, 320, 0, true, 20, 16, 16),  // CTA pairs on 5120-8192-long columns first: fewer
    GBFFT_CLUSTER(10240, 2, 320, 4, true, 5, 16, 16, 4),  // CTAs per row measured faster (N = 16384: K = 2 at
    GBFFT_CLUSTER(10240, 4, 160, 5, true, 5, 16, 16, 2),  // 0.86x the two passes, K = 4 at 0.80x)
    GBFFT_CLUSTER(12288, 2, 384, 0, true, 24, 16, 16),
    GBFFT_CLUSTER(12288, 2, 384, 4, true, 3, 16, 16, 8),
    GBFFT_CLUSTER(12288, 4, 192, 5, true, 24, 8, 16),
    GBFFT_CLUSTER(12288, 4, 192, 4, true, 3, 16, 16, 4),
    GBFFT_CLUSTER(14336, 2, 448, 0, true, 28, 16, 16),
    GBFFT_CLUSTER(14336, 2, 448, 4, true, 7, 16, 16, 4),
    GBFFT_CLUSTER(14336, 4, 256, 0, false, 14, 16, 16),
    GBFFT_CLUSTER(14336, 4, 224, 4, true, 7, 16, 16, 2),
    GBFFT_CLUSTER2(16384, 2, 256, 4, false, 32, 16, 16),  // two butterflies per thread: 0.92x (512 threads: 0.86x)
    GBFFT_CLUSTER(16384, 2, 512, 4, false, 16, 16, 16, 2),
    GBFFT_CLUSTER(16384, 2, 512, 4, false, 32, 16, 16),
    GBFFT_CLUSTER(16384, 4, 256, 4, true, 16, 16, 16),
    GBFFT_CLUSTER(16384, 8, 128, 4, true, 16, 16, 8),
    GBFFT_CLUSTER(20480, 4, 320, 4, true, 5, 16, 16, 4),
    GBFFT_CLUSTER(20480, 8, 160, 5, true, 5, 16, 16, 2),
    GBFFT_CLUSTER(24576, 4, 384, 4, true, 3, 16, 16, 8),
    GBFFT_CLUSTER(24576, 8, 192, 4, true, 3, 16, 16, 4),
    GBFFT_CLUSTER(28672, 4, 448, 4, true, 7, 16, 16, 4),
    GBFFT_CLUSTER(28672, 8, 224, 4, true, 7, 16, 16, 2),
    GBFFT_CLUSTER(32768, 4, 512, 4, true, 16, 16, 16, 2),
    GBFFT_CLUSTER(32768, 8, 256, 4, true, 16, 16, 16),
};

}  // namespace

// Lengths whose default plan is the cluster kernel (variant 0) rather than Eq. 2 as two passes:
// where it measured faster on GB300 (2^26 points): on a CTA pair, 5120 1.18x the two passes, 6144
// 1.11x, 7168 1.08x, 8192 1.06x, 10240 1.07x.  At 12288 / 14336 / 16384 the best cluster variants
// reach 0.95x / 1.01x / 0.92x, so the two passes stay the default.
bool cluster_is_default(int64_t n) { return n == 5120 || n == 6144 || n == 7168 || n == 8192 || n == 10240; }

int cluster_variants_for(int64_t n, const RowsVariant** out, int max_out) {
    int found = 0;
    for (const RowsVariant& v : kCluster) {
        if (v.n != n) continue;
        if (found < max_out && out) out[found] = &v;
        ++found;
    }
    return found;
}

// Stage blocks of the column schedule (length M = N / K) followed by the
// D^N_M table in the layout post[k*M + j1] = w_N^(j1*k).
gbfft_status alloc_cluster_tables(float2** dst, const RowsVariant& v) {
    const int K = v.radix[v.nstages - 1];
    const int64_t m = v.n / K;
    const int cnt = stage_twiddle_count(v.radix, v.nstages - 1);
    if (cudaMalloc(dst, sizeof(float2) * ((size_t)cnt + (size_t)v.n)) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return GBFFT_ERR_OOM;
    }
    if (launch_stage_twiddles(*dst, m, v.radix, v.nstages - 1, 0) != cudaSuccess ||
        launch_post_twiddles(*dst + cnt, v.n, m, 0) != cudaSuccess)
        return GBFFT_ERR_CUDA;
    return GBFFT_OK;
}

}  // namespace gbfft
