// Single-pass variants for lengths p * 2^k (p = 3, 5, 7) up to 4096: one
// radix-p stage first, then power-of-two stages.  E is a multiple of every
// radix in the schedule.
#include "variants.cuh"

namespace gbfft {

static const RowsVariant kMixed[] = {
    GBFFT_ROWS(3, 3, 128, 0, 3),
    GBFFT_ROWS(6, 6, 128, 4, 3, 2),
    GBFFT_ROWS(12, 12, 64, 4, 3, 4),
    GBFFT_ROWS(24, 24, 64, 4, 3, 8),
    GBFFT_ROWS(48, 12, 16, 4, 3, 4, 4),
    GBFFT_ROWS(96, 24, 16, 4, 3, 8, 4),
    GBFFT_ROWS(192, 24, 8, 4, 3, 8, 8),
    GBFFT_ROWS(384, 24, 4, 4, 3, 8, 4, 4),
    GBFFT_ROWS(768, 24, 2, 4, 3, 8, 8, 4),
    GBFFT_ROWS(1536, 24, 2, 4, 3, 8, 8, 8),
    GBFFT_ROWS(3072, 24, 1, 4, 3, 8, 8, 8, 2),
    GBFFT_ROWS(5, 5, 128, 0, 5),
    GBFFT_ROWS(10, 10, 128, 4, 5, 2),
    GBFFT_ROWS(20, 20, 64, 4, 5, 4),
    GBFFT_ROWS(40, 40, 64, 4, 5, 8),
    GBFFT_ROWS(80, 20, 16, 4, 5, 4, 4),
    GBFFT_ROWS(160, 40, 16, 4, 5, 8, 4),
    GBFFT_ROWS(320, 40, 8, 4, 5, 8, 8),
    GBFFT_ROWS(640, 40, 4, 4, 5, 8, 4, 4),
    GBFFT_ROWS(1280, 40, 2, 4, 5, 8, 8, 4),
    GBFFT_ROWS(2560, 40, 2, 4, 5, 8, 8, 8),
    GBFFT_ROWS(7, 7, 128, 0, 7),
    GBFFT_ROWS(14, 14, 128, 4, 7, 2),
    GBFFT_ROWS(28, 28, 64, 4, 7, 4),
    GBFFT_ROWS(56, 56, 32, 4, 7, 8),
    GBFFT_ROWS(112, 28, 16, 4, 7, 4, 4),
    GBFFT_ROWS(224, 56, 16, 4, 7, 8, 4),
    GBFFT_ROWS(448, 56, 8, 4, 7, 8, 8),
    GBFFT_ROWS(896, 56, 4, 4, 7, 8, 4, 4),
    GBFFT_ROWS(1792, 56, 2, 4, 7, 8, 8, 4),
    GBFFT_ROWS(3584, 56, 2, 4, 7, 8, 8, 8),
};

const RowsVariant* rows_variants_mixed(int* count) {
    *count = (int)(sizeof(kMixed) / sizeof(kMixed[0]));
    return kMixed;
}

}  // namespace gbfft
