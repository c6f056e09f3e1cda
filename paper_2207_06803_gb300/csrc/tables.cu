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

cudaError_t launch_twiddle_table(float2* tw, int64_t n, cudaStream_t stream) {
    const int tpb = 256;
    const long long blocks = (n + tpb - 1) / tpb;
    k_twiddle_table<<<(unsigned)blocks, tpb, 0, stream>>>(tw, (long long)n);
    return cudaGetLastError();
}

}  // namespace gbfft
