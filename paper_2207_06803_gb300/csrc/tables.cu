// Twiddle table generation (the only FP64 arithmetic on the GPU).
//
// tw[j] = w_N^j = exp(-2*pi*i*j/N), j < N: the entries of every twiddle
// diagonal D of the schedule (Eq. 2) are powers of w_N, so one table per plan
// serves all stages.  Each entry is evaluated directly (no recurrence) with
// FP64 sincospi on the reduced argument 2j/N in [0, 2), then rounded once to
// float32.
#include "internal.h"

namespace gbfft {

__global__ void k_twiddle_table(float2* tw, long long n) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        double s, c;
        sincospi(2.0 * (double)j / (double)n, &s, &c);
        tw[j] = make_float2((float)c, (float)(-s));
    }
}

// Stage blocks: for each stage s >= 2 of the schedule (L = R_1..R_{s-1} > 1),
// entry (q-1)*L + k of its block is w_N^(q*k*N/(L*R)), q in [1, R), k < L;
// rounded once to float2 (FP32 path) or stored as double2 (FP64 path).
struct ScheduleArg {
    int nstages;
    int radix[kMaxStages];
};

template <class C>
__global__ void k_stage_twiddles(C* tw, long long n, ScheduleArg sch, int total) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int off = 0;
    long long L = 1;
    for (int s = 0; s < sch.nstages; ++s) {
        const int R = sch.radix[s];
        if (L > 1) {
            const int sz = (R - 1) * (int)L;
            if (idx < off + sz) {
                const int i = idx - off;
                const long long q = i / L + 1, k = i % L;
                const long long e = (q * k * (n / (L * R))) % n;
                double sn, cs;
                sincospi(2.0 * (double)e / (double)n, &sn, &cs);
                if constexpr (sizeof(C) == sizeof(float2))
                    tw[idx] = C{(float)cs, (float)(-sn)};
                else
                    tw[idx] = C{cs, -sn};
                return;
            }
            off += sz;
        }
        L *= R;
    }
}

int stage_twiddle_count(const int* radix, int nstages) {
    int total = 0;
    long long L = 1;
    for (int s = 0; s < nstages; ++s) {
        if (L > 1) total += (radix[s] - 1) * (int)L;
        L *= radix[s];
    }
    return total;
}

template <class C>
static cudaError_t stage_twiddles(C* tw, int64_t n, const int* radix, int nstages, cudaStream_t stream) {
    ScheduleArg sch{};
    sch.nstages = nstages;
    for (int s = 0; s < nstages && s < kMaxStages; ++s) sch.radix[s] = radix[s];
    const int total = stage_twiddle_count(radix, nstages);
    if (total == 0) return cudaSuccess;
    const int tpb = 256;
    k_stage_twiddles<C><<<(total + tpb - 1) / tpb, tpb, 0, stream>>>(tw, (long long)n, sch, total);
    return cudaGetLastError();
}

cudaError_t launch_stage_twiddles(float2* tw, int64_t n, const int* radix, int nstages, cudaStream_t stream) {
    return stage_twiddles(tw, n, radix, nstages, stream);
}

cudaError_t launch_stage_twiddles64(double2* tw, int64_t n, const int* radix, int nstages, cudaStream_t stream) {
    return stage_twiddles(tw, n, radix, nstages, stream);
}

__global__ void k_post_twiddles(float2* post, long long n, long long m) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const long long k = idx / m, j1 = idx % m;
    const long long e = (j1 * k) % n;
    double sn, cs;
    sincospi(2.0 * (double)e / (double)n, &sn, &cs);
    post[idx] = make_float2((float)cs, (float)(-sn));
}

cudaError_t launch_post_twiddles(float2* post, int64_t n, int64_t m, cudaStream_t stream) {
    const int tpb = 256;
    k_post_twiddles<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, stream>>>(post, (long long)n, (long long)m);
    return cudaGetLastError();
}

cudaError_t launch_twiddle_table(float2* tw, int64_t n, cudaStream_t stream) {
    const int tpb = 256;
    const long long blocks = (n + tpb - 1) / tpb;
    k_twiddle_table<<<(unsigned)blocks, tpb, 0, stream>>>(tw, (long long)n);
    return cudaGetLastError();
}

}  // namespace gbfft
