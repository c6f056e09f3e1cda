// Single-pass variants for power-of-two lengths 2 .. 4096.  The first entry
// for each length is the planner's default; the others are alternatives the
// autotuner may pick.  GBFFT_ROWS(N, E, T, PS, radices...): E complex per
// thread, T rows per CTA, shared-memory padding shift PS.
#include "variants.cuh"

namespace gbfft {

static const RowsVariant kPow2[] = {
    GBFFT_ROWS(2, 2, 128, 0, 2),
    GBFFT_ROWS(4, 4, 128, 0, 4),
    GBFFT_SMALL(8, 128),
    GBFFT_SMALL(8, 256),
    GBFFT_ROWS(8, 4, 64, 4, 2, 4),
    GBFFT_SMALL(16, 128),
    GBFFT_SMALL(16, 64),
    GBFFT_ROWS(16, 4, 32, 4, 4, 4),
    GBFFT_SMALL(32, 64),
    GBFFT_ROWS(32, 8, 32, 4, 4, 8),
    GBFFT_SMALL(32, 128),
    GBFFT_ROWS(64, 8, 16, 4, 8, 8),
    GBFFT_ROWS(64, 16, 32, 4, 4, 16),
    GBFFT_ROWS(128, 16, 16, 4, 8, 16),
    GBFFT_ROWS(128, 8, 8, 4, 2, 8, 8),
    GBFFT_ROWS(256, 16, 8, 4, 16, 16),
    GBFFT_ROWS(256, 8, 4, 4, 4, 8, 8),
    GBFFT_ROWS(512, 16, 4, 4, 2, 16, 16),
    GBFFT_ROWS(512, 8, 2, 4, 8, 8, 8),
    GBFFT_ROWS_PF(512, 8, 2, 4, 8, 8, 8),
    GBFFT_ROWS(1024, 16, 2, 4, 4, 16, 16),
    GBFFT_ROWS(1024, 16, 2, 4, 16, 16, 4),
    GBFFT_ROWS_PF(1024, 16, 2, 4, 16, 16, 4),
    GBFFT_ROWS(2048, 16, 1, 4, 16, 16, 8),
    GBFFT_ROWS_TMA(2048, 128, 1, 4, 16, 16, 8),
    GBFFT_ROWS(2048, 64, 2, 4, 32, 64),
    GBFFT_ROWS(2048, 16, 2, 4, 8, 16, 16),
    GBFFT_ROWS_PF(2048, 16, 2, 4, 16, 16, 8),
    GBFFT_ROWS(4096, 16, 1, 4, 16, 16, 16),
    GBFFT_ROWS_TMA(4096, 256, 1, 4, 16, 16, 16),
    GBFFT_ROWS(4096, 64, 1, 4, 64, 64),
    GBFFT_ROWS(4096, 64, 2, 4, 64, 64),
    GBFFT_ROWS_PF(4096, 16, 1, 4, 16, 16, 16),
    GBFFT_ROWS(4096, 8, 1, 4, 8, 8, 8, 8),
};

const RowsVariant* rows_variants_pow2(int* count) {
    *count = (int)(sizeof(kPow2) / sizeof(kPow2[0]));
    return kPow2;
}

}  // namespace gbfft
