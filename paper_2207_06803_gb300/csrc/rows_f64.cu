// Complex128 single-pass variants (FP64 arithmetic, double2 I/O and stage
// twiddles): every length 2^k, 3*2^k, 5*2^k, 7*2^k up to 4096.  Each thread
// holds at most 16 complex doubles per stage; radix-16 stages are preferred
// because they need the fewest FP64 operations per point (the FP64 pipe, not
// HBM, bounds this path on GB300).  One radix-p stage comes first for mixed
// lengths; the thread count is sized by the power-of-two stages.  Where a
// composite first stage (DFT_6, 10, 12, 14 by the prime-factor map) fits in 16
// complex per thread and saves a stage, it is the default (5-10 % more GFLOP/s:
// no twiddles inside it, one exchange fewer); the first entry of a length is its
// default, the second the radix-p-first alternative.
#include "variants.cuh"

#define GBFFT_ROWS_D(N, TPB, T, PS, ...) ::gbfft::make_rows_d_variant<N, TPB, T, PS, __VA_ARGS__>()

namespace gbfft {

static const RowsVariant kF64[] = {
    GBFFT_ROWS_D(2, 256, 256, 0, 2),
    GBFFT_ROWS_D(4, 256, 256, 0, 4),
    GBFFT_ROWS_D(8, 128, 64, 4, 2, 4),
    GBFFT_ROWS_D(16, 256, 64, 4, 4, 4),
    GBFFT_ROWS_D(32, 128, 32, 4, 4, 8),
    GBFFT_ROWS_D(64, 128, 16, 4, 8, 8),
    GBFFT_ROWS_D(128, 128, 16, 4, 8, 16),
    GBFFT_ROWS_D(256, 64, 4, 4, 16, 16),
    GBFFT_ROWS_D(512, 64, 2, 4, 2, 16, 16),
    GBFFT_ROWS_D(1024, 64, 1, 4, 4, 16, 16),
    GBFFT_ROWS_D(2048, 128, 1, 4, 8, 16, 16),
    GBFFT_ROWS_D(4096, 256, 1, 4, 16, 16, 16),
    GBFFT_ROWS_D(3, 256, 256, 0, 3),
    GBFFT_ROWS_D(6, 256, 128, 0, 3, 2),
    GBFFT_ROWS_D(12, 128, 64, 0, 3, 4),
    GBFFT_ROWS_D(24, 64, 32, 0, 3, 8),
    GBFFT_ROWS_D(48, 64, 16, 4, 3, 16),
    GBFFT_ROWS_D(96, 64, 8, 0, 6, 16),
    GBFFT_ROWS_D(96, 64, 8, 4, 3, 2, 16),
    GBFFT_ROWS_D(192, 64, 4, 0, 12, 16),
    GBFFT_ROWS_D(192, 64, 4, 0, 3, 4, 16),
    GBFFT_ROWS_D(384, 64, 2, 0, 3, 8, 16),
    GBFFT_ROWS_D(768, 64, 1, 4, 3, 16, 16),
    GBFFT_ROWS_D(1536, 128, 1, 0, 6, 16, 16),
    GBFFT_ROWS_D(1536, 128, 1, 4, 3, 16, 16, 2),
    GBFFT_ROWS_D(3072, 256, 1, 0, 12, 16, 16),
    GBFFT_ROWS_D(3072, 256, 1, 4, 3, 16, 16, 4),
    GBFFT_ROWS_D(5, 256, 256, 0, 5),
    GBFFT_ROWS_D(10, 256, 128, 0, 5, 2),
    GBFFT_ROWS_D(20, 128, 64, 0, 5, 4),
    GBFFT_ROWS_D(40, 64, 16, 0, 5, 8),
    GBFFT_ROWS_D(80, 64, 8, 0, 5, 16),
    GBFFT_ROWS_D(160, 64, 4, 0, 10, 16),
    GBFFT_ROWS_D(160, 64, 4, 0, 5, 2, 16),
    GBFFT_ROWS_D(320, 64, 2, 0, 5, 4, 16),
    GBFFT_ROWS_D(640, 64, 1, 0, 5, 8, 16),
    GBFFT_ROWS_D(1280, 96, 1, 4, 5, 16, 16),
    GBFFT_ROWS_D(2560, 256, 1, 0, 10, 16, 16),
    GBFFT_ROWS_D(2560, 192, 1, 4, 5, 16, 16, 2),
    GBFFT_ROWS_D(7, 256, 256, 0, 7),
    GBFFT_ROWS_D(14, 256, 128, 0, 7, 2),
    GBFFT_ROWS_D(28, 64, 32, 0, 7, 4),
    GBFFT_ROWS_D(56, 64, 16, 0, 7, 8),
    GBFFT_ROWS_D(112, 64, 8, 0, 7, 16),
    GBFFT_ROWS_D(224, 64, 4, 0, 14, 16),
    GBFFT_ROWS_D(224, 64, 4, 0, 7, 2, 16),
    GBFFT_ROWS_D(448, 64, 2, 0, 7, 4, 16),
    GBFFT_ROWS_D(896, 64, 1, 0, 7, 8, 16),
    GBFFT_ROWS_D(1792, 128, 1, 4, 7, 16, 16),
    GBFFT_ROWS_D(3584, 256, 1, 0, 14, 16, 16),
    GBFFT_ROWS_D(3584, 256, 1, 4, 7, 16, 16, 2),
};

const RowsVariant* rows_variants_f64(int* count) {
    *count = (int)(sizeof(kF64) / sizeof(kF64[0]));
    return kF64;
}

int rows_variants_f64_for(int64_t n, const RowsVariant** out, int max_out) {
    int found = 0;
    for (const RowsVariant& v : kF64) {
        if (v.n != n) continue;
        if (found < max_out && out) out[found] = &v;
        ++found;
    }
    return found;
}

}  // namespace gbfft
