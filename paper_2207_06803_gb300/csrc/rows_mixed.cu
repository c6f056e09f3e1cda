// Single-pass variants for lengths p * 2^k (p = 3, 5, 7) up to 4096.  The
// first entry of each length is its default.  From 10 to 48 that is the
// one-row-per-thread kernel (GBFFT_SMALL2); from 56 up, a GBFFT_ROWS_T schedule
// (explicit thread count; a stage whose butterflies do not divide the threads
// runs ceil(butterflies/threads) per thread, guarded) whose first stage is a
// composite p * 2^j codelet.  Schedules with a lone radix-p stage first and the
// GBFFT_ROWS entries (E a multiple of every radix) remain as alternatives.
// Thread counts, rows per CTA and pad shifts are the fastest measured.
#include "variants.cuh"

namespace gbfft {

static const RowsVariant kMixed[] = {
    // N = 10 ... 48: one row per thread, both Stockham stages in registers, the tile staged through shared
    // memory with 16-byte accesses (the defaults: 6.5-6.8 TB/s against 5.1-6.4 for the tile kernels below)
    GBFFT_SMALL2(10, 128, 5, 2),
    GBFFT_SMALL2(12, 128, 3, 4),
    GBFFT_SMALL2(14, 128, 7, 2),
    GBFFT_SMALL2(20, 128, 5, 4),
    GBFFT_SMALL2(24, 128, 3, 8),
    GBFFT_SMALL2(28, 128, 7, 4),
    GBFFT_SMALL2(40, 64, 5, 8),
    GBFFT_SMALL2(48, 64, 3, 16),
    // N = 56: a tile of 64 rows, DFT_14 (prime-factor) then radix 4 on 256 threads, 6.39 TB/s against 6.10-6.20
    // for one row per thread (56 complex in registers, 166+ registers per thread)
    GBFFT_ROWS_T(56, 256, 64, 0, 14, 4),
    GBFFT_SMALL2(56, 64, 7, 8),
    // N = 4 as two radix-2 stages (Eq. 1's factorisation; an alternative to the radix-4 codelet)
    GBFFT_ROWS(4, 4, 128, 0, 2, 2),
    GBFFT_ROWS(3, 3, 128, 0, 3),
    GBFFT_ROWS(6, 6, 128, 4, 3, 2),
    GBFFT_ROWS_T(6, 768, 256, 0, 3, 2),
    GBFFT_ROWS(12, 12, 64, 4, 3, 4),
    GBFFT_ROWS_T(12, 768, 256, 0, 3, 4),
    GBFFT_ROWS_T(24, 384, 128, 0, 3, 8),
    GBFFT_ROWS(24, 24, 64, 4, 3, 8),
    GBFFT_ROWS(48, 12, 16, 4, 3, 4, 4),
    GBFFT_ROWS_T(48, 192, 64, 4, 3, 16),
    GBFFT_ROWS(5, 5, 128, 0, 5),
    GBFFT_ROWS(10, 10, 128, 4, 5, 2),
    GBFFT_ROWS_T(10, 640, 128, 0, 5, 2),
    GBFFT_ROWS_T(20, 640, 128, 0, 5, 4),
    GBFFT_ROWS(20, 20, 64, 4, 5, 4),
    GBFFT_ROWS_T(40, 320, 64, 0, 5, 8),
    GBFFT_ROWS(40, 40, 64, 4, 5, 8),
    GBFFT_ROWS(7, 7, 128, 0, 7),
    GBFFT_ROWS(14, 14, 128, 4, 7, 2),
    GBFFT_ROWS_T(14, 896, 128, 0, 7, 2),
    GBFFT_ROWS(28, 28, 64, 4, 7, 4),
    GBFFT_ROWS_T(28, 896, 128, 0, 7, 4),
    GBFFT_ROWS(56, 56, 32, 4, 7, 8),
    GBFFT_ROWS_T(56, 448, 64, 0, 7, 8),

    // N = 80 ... 3584: the default (first) schedule of each length opens with a composite stage
    // p * 2^j (DFT_6 ... DFT_56 by the prime-factor map, no twiddles inside) and continues with
    // radix-8/16/32 stages, three stages at most, so that every stage fills the CTA's threads: 95-102 %
    // of measured HBM against 75-96 % for the radix-p-first schedules kept after it as alternatives
    // (a lone radix-p stage spreads N/p butterflies unevenly over threads sized for radix 16, and lengths
    // above 1024 needed a fourth, radix-2/4 stage).
    GBFFT_ROWS_T(96, 128, 16, 0, 12, 8),
    GBFFT_ROWS_T(96, 128, 16, 0, 6, 16),
    GBFFT_ROWS_T(96, 192, 32, 4, 3, 2, 16),
    GBFFT_ROWS(96, 24, 16, 4, 3, 8, 4),
    GBFFT_ROWS_T(192, 256, 16, 0, 12, 16),
    GBFFT_ROWS_T(192, 192, 16, 0, 3, 4, 16),
    GBFFT_ROWS(192, 24, 8, 4, 3, 8, 8),
    GBFFT_ROWS_T(384, 192, 8, 4, 24, 16),
    GBFFT_ROWS_T(384, 192, 8, 0, 3, 8, 16),
    GBFFT_ROWS(384, 24, 4, 4, 3, 8, 4, 4),
    GBFFT_ROWS_T(768, 128, 2, 0, 6, 8, 16),
    GBFFT_ROWS_T(768, 192, 4, 4, 3, 16, 16),
    GBFFT_ROWS(768, 24, 2, 4, 3, 8, 8, 4),
    GBFFT_ROWS_T(1536, 128, 1, 0, 6, 16, 16),
    GBFFT_ROWS_T(1536, 192, 2, 4, 3, 16, 16, 2),
    GBFFT_ROWS_TMA(1536, 192, 2, 4, 3, 16, 16, 2),
    GBFFT_ROWS(1536, 24, 2, 4, 3, 8, 8, 8),
    GBFFT_ROWS_T(3072, 192, 1, 5, 24, 8, 16),
    GBFFT_ROWS_T(3072, 256, 1, 0, 12, 16, 16),
    GBFFT_ROWS_T(3072, 192, 1, 4, 3, 16, 16, 4),
    GBFFT_ROWS_TMA(3072, 192, 1, 4, 3, 16, 16, 4),
    GBFFT_ROWS_T(80, 160, 16, 0, 10, 8),
    GBFFT_ROWS_T(80, 160, 32, 5, 5, 16),
    GBFFT_ROWS(80, 20, 16, 4, 5, 4, 4),
    GBFFT_ROWS_T(160, 128, 8, 0, 10, 16),
    GBFFT_ROWS_T(160, 160, 8, 0, 20, 8),
    GBFFT_ROWS_T(160, 160, 16, 0, 5, 2, 16),
    GBFFT_ROWS(160, 40, 16, 4, 5, 8, 4),
    GBFFT_ROWS_T(320, 160, 8, 0, 20, 16),
    GBFFT_ROWS_T(320, 160, 8, 0, 5, 4, 16),
    GBFFT_ROWS(320, 40, 8, 4, 5, 8, 8),
    // 640: the radix-5-first schedule stays the default (100 % of HBM; DFT_40 first: 79 %)
    GBFFT_ROWS_T(640, 160, 4, 0, 5, 8, 16),
    GBFFT_ROWS_T(640, 128, 4, 0, 20, 32),
    GBFFT_ROWS(640, 40, 4, 4, 5, 8, 4, 4),
    GBFFT_ROWS_T(1280, 160, 1, 0, 10, 8, 16),
    GBFFT_ROWS_T(1280, 160, 2, 5, 5, 16, 16),
    GBFFT_ROWS(1280, 40, 2, 4, 5, 8, 8, 4),
    GBFFT_ROWS_T(2560, 160, 1, 0, 20, 8, 16),
    GBFFT_ROWS_T(2560, 160, 1, 0, 10, 16, 16),
    GBFFT_ROWS_T(2560, 160, 1, 5, 5, 16, 16, 2),
    GBFFT_ROWS_TMA(2560, 160, 1, 5, 5, 16, 16, 2),
    GBFFT_ROWS(2560, 40, 2, 4, 5, 8, 8, 8),
    GBFFT_ROWS_T(112, 112, 8, 0, 14, 8),
    GBFFT_ROWS_T(112, 224, 32, 4, 7, 16),
    GBFFT_ROWS(112, 28, 16, 4, 7, 4, 4),
    GBFFT_ROWS_T(224, 128, 8, 0, 14, 16),
    GBFFT_ROWS_T(224, 224, 16, 0, 7, 2, 16),
    GBFFT_ROWS(224, 56, 16, 4, 7, 8, 4),
    GBFFT_ROWS_T(448, 224, 8, 0, 28, 16),
    GBFFT_ROWS_T(448, 224, 8, 0, 7, 4, 16),
    GBFFT_ROWS(448, 56, 8, 4, 7, 8, 8),
    GBFFT_ROWS_T(896, 128, 4, 0, 28, 32),
    GBFFT_ROWS_T(896, 224, 4, 0, 7, 8, 16),
    GBFFT_ROWS(896, 56, 4, 4, 7, 8, 4, 4),
    GBFFT_ROWS_T(1792, 128, 1, 0, 14, 8, 16),
    GBFFT_ROWS_T(1792, 224, 2, 4, 7, 16, 16),
    GBFFT_ROWS(1792, 56, 2, 4, 7, 8, 8, 4),
    GBFFT_ROWS_T(3584, 256, 1, 0, 14, 16, 16),
    GBFFT_ROWS_T(3584, 224, 1, 4, 7, 16, 16, 2),
    GBFFT_ROWS_TMA(3584, 224, 1, 4, 7, 16, 16, 2),
    GBFFT_ROWS(3584, 56, 2, 4, 7, 8, 8, 8),
};

const RowsVariant* rows_variants_mixed(int* count) {
    *count = (int)(sizeof(kMixed) / sizeof(kMixed[0]));
    return kMixed;
}

}  // namespace gbfft
