// Internal declarations shared by the library's translation units (not part
// of the public C ABI in include/gbfft.h).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "gbfft.h"

namespace gbfft {

constexpr int kMaxStages = 8;

// One compiled single-pass kernel (both directions) for transform length n.
struct RowsVariant {
    int n;                  // transform length
    int e;                  // complex elements each thread holds per stage
    int rows;               // transforms per CTA
    int tpb;                // threads per CTA
    int ps;                 // shared-memory padding shift (0 = none)
    int nstages;            // schedule length
    int radix[kMaxStages];  // R_1 .. R_t
    int smem;               // dynamic shared memory, bytes
    const void* kfwd;       // __global__ k_stockham_rows<..., S = -1, ...>
    const void* kinv;       // __global__ k_stockham_rows<..., S = +1, ...>
};

// Per-translation-unit variant tables, gathered by the registry in api.cu.
const RowsVariant* rows_variants_pow2(int* count);
const RowsVariant* rows_variants_mixed(int* count);

// All variants for length n, in preference order (the first is the default).
int rows_variants_for(int64_t n, const RowsVariant** out, int max_out);

// Launch a rows variant over `batch` contiguous rows.
cudaError_t launch_rows(const RowsVariant& v, int direction, const float2* in, float2* out, const float2* tw,
                        long long batch, cudaStream_t stream);

// tw[j] = exp(-2*pi*i*j/n) for j < n, evaluated in FP64 on the device.
cudaError_t launch_twiddle_table(float2* tw, int64_t n, cudaStream_t stream);

}  // namespace gbfft
