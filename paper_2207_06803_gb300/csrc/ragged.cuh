// Ragged batches: thousands of transforms of uneven lengths in one persistent launch.
//
// The host groups the transforms by length ("class"), cuts each group into
// work items of at most T_c rows (the tile shape of class c, chosen by the
// autotuner), orders the items longest-first and uploads them with the list of
// row offsets.  Each CTA of the persistent kernel repeatedly claims the next
// item with one atomic increment and runs the class's Stockham schedule on it
// (the same stage code as the single-pass kernel, with per-row offsets held in
// shared memory), until the queue is empty.  Every class uses 256 threads per
// CTA, so one kernel serves all classes.
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

// (class index, N, T rows per full tile, shared-memory pad shift, radix
// schedule...).  Every class runs kRaggedThreads threads; T is about
// 4096/N (at most 256) so a tile holds ~4096 elements and each thread at most
// 32 complex values; a stage with fewer butterflies than threads leaves some
// idle.
#define GBFFT_RAGGED_CLASSES(X)               \
    X(0, 8, 256, 4, 2, 4)                     \
    X(1, 10, 256, 0, 5, 2)                    \
    X(2, 12, 256, 0, 3, 4)                    \
    X(3, 14, 256, 0, 7, 2)                    \
    X(4, 16, 256, 4, 4, 4)                    \
    X(5, 20, 204, 0, 5, 4)                    \
    X(6, 24, 170, 0, 3, 8)                    \
    X(7, 28, 146, 0, 7, 4)                    \
    X(8, 32, 128, 4, 4, 8)                    \
    X(9, 40, 102, 0, 5, 8)                    \
    X(10, 48, 85, 4, 3, 16)                   \
    X(11, 56, 73, 0, 7, 8)                    \
    X(12, 64, 64, 4, 8, 8)                    \
    X(13, 80, 51, 5, 5, 16)                   \
    X(14, 96, 42, 4, 3, 2, 16)                \
    X(15, 112, 36, 4, 7, 16)                  \
    X(16, 128, 32, 4, 8, 16)                  \
    X(17, 160, 25, 0, 5, 2, 16)               \
    X(18, 192, 21, 0, 3, 4, 16)               \
    X(19, 224, 18, 0, 7, 2, 16)               \
    X(20, 256, 16, 4, 16, 16)                 \
    X(21, 320, 12, 0, 5, 4, 16)               \
    X(22, 384, 10, 0, 3, 8, 16)               \
    X(23, 448, 9, 0, 7, 4, 16)                \
    X(24, 512, 8, 4, 2, 16, 16)               \
    X(25, 640, 6, 0, 5, 8, 16)                \
    X(26, 768, 5, 4, 3, 16, 16)               \
    X(27, 896, 4, 0, 7, 8, 16)                \
    X(28, 1024, 4, 4, 4, 16, 16)              \
    X(29, 1280, 3, 5, 5, 16, 16)              \
    X(30, 1536, 2, 4, 3, 16, 16, 2)           \
    X(31, 1792, 2, 4, 7, 16, 16)              \
    X(32, 2048, 2, 4, 16, 16, 8)              \
    X(33, 2560, 1, 5, 5, 16, 16, 2)           \
    X(34, 3072, 1, 4, 3, 16, 16, 4)           \
    X(35, 3584, 1, 4, 7, 16, 16, 2)           \
    X(36, 4096, 1, 4, 16, 16, 16)             \
    X(37, 5120, 1, 4, 5, 16, 16, 4)           \
    X(38, 6144, 1, 4, 3, 16, 16, 8)           \
    X(39, 7168, 1, 4, 7, 16, 16, 4)           \
    X(40, 8192, 1, 4, 16, 16, 32)

constexpr int kRaggedClasses = 41;

}  // namespace gbfft
