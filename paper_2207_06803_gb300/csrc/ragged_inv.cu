// Inverse-direction instantiation of the ragged persistent kernel.
#include "internal.h"
#include "ragged.cuh"

namespace gbfft {

template __global__ void k_ragged<+1>(const float2*, float2*, const RaggedItem*, int, const long long*,
                                      const RaggedLen* __restrict__, const float2* __restrict__, int*,
                                      const int* __restrict__, int*,
                                      long long);

const void* ragged_kernel_inv() { return (const void*)&k_ragged<+1>; }

}  // namespace gbfft
