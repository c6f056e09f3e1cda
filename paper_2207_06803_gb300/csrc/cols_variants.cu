// Column-transform variants for the two passes of Eq. 2 (see columns.cuh).
// Every entry uses C = 16 columns per CTA, so a split N = K * M is available
// whenever both K and M are registered lengths.
#include "columns.cuh"
#include "internal.h"

namespace gbfft {

template <int LEN, int E, int C, int... Rs>
inline ColsVariant make_cols_variant() {
    static_assert(((Rs * ...) == LEN), "radix schedule must multiply to the column length");
    static_assert((C * LEN) % E == 0, "tile must split evenly over threads");
    return ColsVariant{LEN,
                       E,
                       C,
                       C * LEN / E,
                       (int)sizeof...(Rs),
                       {Rs...},
                       (int)(LEN * (C + 1) * sizeof(float2)),
                       (const void*)&k_stockham_cols<LEN, -1, E, C, kColsPass1, Rs...>,
                       (const void*)&k_stockham_cols<LEN, +1, E, C, kColsPass1, Rs...>,
                       (const void*)&k_stockham_cols<LEN, -1, E, C, kColsPass2, Rs...>,
                       (const void*)&k_stockham_cols<LEN, +1, E, C, kColsPass2, Rs...>};
}

#define GBFFT_COLS(LEN, E, C, ...) make_cols_variant<LEN, E, C, __VA_ARGS__>()

static const ColsVariant kCols[] = {
    GBFFT_COLS(8, 4, 16, 2, 4),
    GBFFT_COLS(16, 4, 16, 4, 4),
    GBFFT_COLS(32, 8, 16, 4, 8),
    GBFFT_COLS(48, 12, 16, 3, 4, 4),
    GBFFT_COLS(64, 8, 16, 8, 8),
    GBFFT_COLS(80, 20, 16, 5, 4, 4),
    GBFFT_COLS(96, 24, 16, 3, 8, 4),
    GBFFT_COLS(112, 28, 16, 7, 4, 4),
    GBFFT_COLS(128, 16, 16, 8, 16),
    GBFFT_COLS(256, 16, 16, 16, 16),
    // 512: two radix-16 butterflies per thread (512 threads, 62-64 registers: two CTAs per SM); the form with
    // one radix-8 butterfly per thread (1024 threads, one CTA per SM) ran 16-29 % slower (N = 131072: 2.58 against
    // 3.12 TB/s; 512 x 1024: 2.44 against 3.15)
    GBFFT_COLS(512, 16, 16, 16, 16, 2),
};

const ColsVariant* cols_variant_for(int64_t len) {
    for (const ColsVariant& v : kCols)
        if (v.len == len) return &v;
    return nullptr;
}

// Short column lengths for the multi-dimensional plans' axis passes: 64 columns per
// CTA (128 or 256 threads instead of 32 or 64, so that an SM holds enough loads in
// flight), used where the axis's row stride is a multiple of 64.
static const ColsVariant kColsWide[] = {
    GBFFT_COLS(8, 4, 64, 2, 4),
    GBFFT_COLS(16, 4, 64, 4, 4),
};

const ColsVariant* cols_variant_for_nd(int64_t len, int64_t ncols) {
    for (const ColsVariant& v : kColsWide)
        if (v.len == len && ncols % v.c == 0) return &v;
    return cols_variant_for(len);
}

const ColsVariant* cols_variants(int* count) {
    *count = (int)(sizeof(kCols) / sizeof(kCols[0]));
    return kCols;
}

cudaError_t prepare_cols(const ColsVariant& v) {
    if (v.smem <= 48 * 1024) return cudaSuccess;
    const void* ks[4] = {v.k1f, v.k1i, v.k2f, v.k2i};
    for (const void* k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_cols(const ColsVariant& v, int pass, int direction, const float2* in, float2* out,
                        const float2* tw, const float2* post, long long batch, int ncols, cudaStream_t stream) {
    if (batch <= 0) return cudaSuccess;
    const long long blocks = batch * (ncols / v.c);
    void* args[] = {(void*)&in, (void*)&out, (void*)&tw, (void*)&post, (void*)&ncols};
    const void* fn = pass == 1 ? (direction == GBFFT_FORWARD ? v.k1f : v.k1i)
                               : (direction == GBFFT_FORWARD ? v.k2f : v.k2i);
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(v.tpb), args, (size_t)v.smem, stream);
}

}  // namespace gbfft
