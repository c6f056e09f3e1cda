// Helpers to declare single-pass kernel variants as table entries.
#pragma once
#include "internal.h"
#include "stockham.cuh"

namespace gbfft {

template <int N, int E, int T, int PS, int... Rs>
inline RowsVariant make_rows_variant() {
    static_assert(((Rs * ...) == N), "radix schedule must multiply to N");
    static_assert((T * N) % E == 0, "tile must split evenly over threads");
    return RowsVariant{kRowsDirect,
                       N,
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

template <int N, int E, int T, int PS, int... Rs>
inline RowsVariant make_rows_pf_variant() {
    static_assert(((Rs * ...) == N), "radix schedule must multiply to N");
    static_assert((T * N) % E == 0, "tile must split evenly over threads");
    return RowsVariant{kRowsPersistent,
                       N,
                       E,
                       T,
                       T * N / E,
                       PS,
                       (int)sizeof...(Rs),
                       {Rs...},
                       (int)(sizeof...(Rs) > 1 ? smem_elems<T, N, PS>() * sizeof(float2) : 0),
                       (const void*)&k_stockham_rows_pf<N, -1, E, T, PS, Rs...>,
                       (const void*)&k_stockham_rows_pf<N, +1, E, T, PS, Rs...>};
}

template <int N, int TPB, int T, int PS, int... Rs>
inline RowsVariant make_rows_t_variant() {
    static_assert(((Rs * ...) == N), "radix schedule must multiply to N");
    return RowsVariant{kRowsDirect,
                       N,
                       capacity_of_r<N, T, TPB, Rs...>(),
                       T,
                       TPB,
                       PS,
                       (int)sizeof...(Rs),
                       {Rs...},
                       (int)(sizeof...(Rs) > 1 ? smem_elems<T, N, PS>() * sizeof(float2) : 0),
                       (const void*)&k_stockham_rows_t<N, -1, TPB, T, PS, Rs...>,
                       (const void*)&k_stockham_rows_t<N, +1, TPB, T, PS, Rs...>};
}

// Complex128 rows (FP64): like make_rows_t_variant with 16-byte elements.
template <int N, int TPB, int T, int PS, int... Rs>
inline RowsVariant make_rows_d_variant() {
    static_assert(((Rs * ...) == N), "radix schedule must multiply to N");
    return RowsVariant{kRowsDirect,
                       N,
                       capacity_of_r<N, T, TPB, Rs...>(),
                       T,
                       TPB,
                       PS,
                       (int)sizeof...(Rs),
                       {Rs...},
                       (int)(sizeof...(Rs) > 1 ? smem_elems<T, N, PS>() * sizeof(double2) : 0),
                       (const void*)&k_stockham_rows_d<N, -1, TPB, T, PS, Rs...>,
                       (const void*)&k_stockham_rows_d<N, +1, TPB, T, PS, Rs...>};
}

template <int N, int TPB, int T, int PS, int... Rs>
inline RowsVariant make_rows_tma_variant() {
    static_assert(((Rs * ...) == N), "radix schedule must multiply to N");
    static_assert((T * N) % 2 == 0, "bulk copies move whole 16-byte units");
    return RowsVariant{kRowsTma,
                       N,
                       capacity_of_r<N, T, TPB, Rs...>(),
                       T,
                       TPB,
                       PS,
                       (int)sizeof...(Rs),
                       {Rs...},
                       tma_smem_bytes<T, N, PS>(),
                       (const void*)&k_stockham_rows_tma<N, -1, TPB, T, PS, Rs...>,
                       (const void*)&k_stockham_rows_tma<N, +1, TPB, T, PS, Rs...>};
}

template <int N, int T>
inline RowsVariant make_small_variant() {
    return RowsVariant{kRowsSmall,
                       N,
                       N,
                       T,
                       T,
                       0,
                       1,
                       {N},
                       (int)(T * (N + 2) * sizeof(float2)),
                       (const void*)&k_stockham_small<N, -1, T>,
                       (const void*)&k_stockham_small<N, +1, T>};
}

// One row per thread, two register-resident Stockham stages (N = R1 * R2).
template <int N, int T, int R1, int R2>
inline RowsVariant make_small2_variant() {
    return RowsVariant{kRowsSmall,
                       N,
                       N,
                       T,
                       T,
                       0,
                       2,
                       {R1, R2},
                       (int)(T * small2_pitch(N) * sizeof(float2)),
                       (const void*)&k_stockham_small2<N, -1, T, R1, R2>,
                       (const void*)&k_stockham_small2<N, +1, T, R1, R2>};
}

}  // namespace gbfft

#define GBFFT_SMALL2(N, T, R1, R2) ::gbfft::make_small2_variant<N, T, R1, R2>()
#define GBFFT_ROWS(N, E, T, PS, ...) ::gbfft::make_rows_variant<N, E, T, PS, __VA_ARGS__>()
#define GBFFT_ROWS_PF(N, E, T, PS, ...) ::gbfft::make_rows_pf_variant<N, E, T, PS, __VA_ARGS__>()
#define GBFFT_SMALL(N, T) ::gbfft::make_small_variant<N, T>()
#define GBFFT_ROWS_T(N, TPB, T, PS, ...) ::gbfft::make_rows_t_variant<N, TPB, T, PS, __VA_ARGS__>()
#define GBFFT_ROWS_TMA(N, TPB, T, PS, ...) ::gbfft::make_rows_tma_variant<N, TPB, T, PS, __VA_ARGS__>()
