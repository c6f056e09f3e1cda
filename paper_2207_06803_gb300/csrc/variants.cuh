// Helpers to declare single-pass kernel variants as table entries.
#pragma once
#include "internal.h"
#include "stockham.cuh"

namespace gbfft {

template <int N, int E, int T, int PS, int... Rs>
inline RowsVariant make_rows_variant() {
    static_assert(((Rs * ...) == N), "radix schedule must multiply to N");
    static_assert((T * N) % E == 0, "tile must split evenly over threads");
    return RowsVariant{N,
                       E,
                       T,
                       T * N / E,
                       PS,
                       (int)sizeof...(Rs),
                       {Rs...},
                       (int)(sizeof...(Rs) > 1 ? smem_elems<T, N, PS>() * sizeof(float2) : 0),
                       (const void*)&k_stockham_rows<N, -1, E, T, PS, Rs...>,
                       (const void*)&k_stockham_rows<N, +1, E, T, PS, Rs...>};
}

}  // namespace gbfft

#define GBFFT_ROWS(N, E, T, PS, ...) ::gbfft::make_rows_variant<N, E, T, PS, __VA_ARGS__>()
