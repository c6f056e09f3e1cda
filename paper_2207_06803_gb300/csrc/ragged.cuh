// Ragged batches: thousands of transforms of uneven lengths in one persistent launch.
//
// The host groups the transforms by length ("class"), cuts each group into
// work items of at most T_c rows (the tile shape of class c, chosen by the
// autotuner), orders the items longest-first and uploads them with the list of
// row offsets.  Each CTA of the persistent kernel repeatedly claims the next
// item with one atomic increment and runs the class's Stockham schedule on it
// (the same stage code as the single-pass kernel, with per-row offsets held in
// shared memory), until the queue is empty.  Every class uses 256 threads per
// CTA (T_c * N_c / E_c = 256), so one kernel serves all classes.
//
// Items carry a `ready` word.  The host publishes all items ready; a CTA that
// claims an item still marked not ready waits for it with a bounded spin
// (globaltimer deadline), and on expiry records GBFFT_ERR_TIMEOUT in the plan's
// status word, skips the item and carries on: no wait in this kernel is
// unbounded.
#pragma once
#include <cuda_runtime.h>

#include "stockham.cuh"

namespace gbfft {

constexpr int kRaggedThreads = 256;

struct RaggedItem {
    int cls;    // class index (length) in the class table
    int count;  // rows in this item (<= T of the class)
    int first;  // index of the item's first row offset in the offset list
    int ready;  // nonzero once the item may be processed
};

// (class index, N, E, shared-memory pad shift, radix schedule...).  T = 256*E/N.
#define GBFFT_RAGGED_CLASSES(X)              \
    X(0, 8, 4, 4, 2, 4)                      \
    X(1, 10, 10, 4, 5, 2)                    \
    X(2, 12, 12, 4, 3, 4)                    \
    X(3, 14, 14, 4, 7, 2)                    \
    X(4, 16, 4, 4, 4, 4)                     \
    X(5, 20, 20, 4, 5, 4)                    \
    X(6, 24, 24, 4, 3, 8)                    \
    X(7, 28, 28, 4, 7, 4)                    \
    X(8, 32, 8, 4, 4, 8)                     \
    X(9, 40, 40, 4, 5, 8)                    \
    X(10, 48, 12, 4, 3, 4, 4)                \
    X(11, 56, 28, 4, 7, 2, 4)                \
    X(12, 64, 8, 4, 8, 8)                    \
    X(13, 80, 20, 4, 5, 4, 4)                \
    X(14, 96, 24, 4, 3, 8, 4)                \
    X(15, 112, 28, 4, 7, 4, 4)               \
    X(16, 128, 16, 4, 8, 16)                 \
    X(17, 160, 40, 4, 5, 8, 4)               \
    X(18, 192, 24, 4, 3, 8, 8)               \
    X(19, 224, 28, 4, 7, 4, 4, 2)            \
    X(20, 256, 16, 4, 16, 16)                \
    X(21, 320, 40, 4, 5, 8, 8)               \
    X(22, 384, 24, 4, 3, 8, 4, 4)            \
    X(23, 448, 28, 4, 7, 4, 4, 4)            \
    X(24, 512, 16, 4, 2, 16, 16)             \
    X(25, 640, 40, 4, 5, 8, 4, 4)            \
    X(26, 768, 24, 4, 3, 8, 8, 4)            \
    X(27, 896, 28, 4, 7, 4, 4, 4, 2)         \
    X(28, 1024, 16, 4, 4, 16, 16)            \
    X(29, 1280, 40, 4, 5, 8, 8, 4)           \
    X(30, 1536, 24, 4, 3, 8, 8, 8)           \
    X(31, 1792, 28, 4, 7, 4, 4, 4, 4)        \
    X(32, 2048, 16, 4, 16, 16, 8)            \
    X(33, 2560, 40, 4, 5, 8, 8, 8)           \
    X(34, 3072, 24, 4, 3, 8, 8, 8, 2)        \
    X(35, 3584, 28, 4, 7, 4, 4, 4, 4, 2)     \
    X(36, 4096, 16, 4, 16, 16, 16)           \
    X(37, 5120, 20, 4, 5, 4, 4, 4, 4, 4)     \
    X(38, 6144, 24, 4, 3, 8, 8, 8, 4)        \
    X(39, 7168, 28, 4, 7, 4, 4, 4, 4, 4)     \
    X(40, 8192, 32, 4, 16, 16, 32)

constexpr int kRaggedClasses = 41;

}  // namespace gbfft
