// Internal declarations shared by the library's translation units (not part
// of the public C ABI in include/gbfft.h).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "gbfft.h"

namespace gbfft {

constexpr int kMaxStages = 8;

enum RowsKind : int {
    kRowsDirect = 0,      // k_stockham_rows: one tile per CTA
    kRowsPersistent = 1,  // k_stockham_rows_pf: resident CTAs walk tiles with register prefetch
    kRowsSmall = 2,       // k_stockham_small: one row per thread, tile staged through shared memory
    kRowsTma = 3,         // k_stockham_rows_tma: persistent, next tile prefetched by TMA bulk copy
    kRowsCluster = 4,     // k_stockham_cluster: one row per cluster of K CTAs (Eq. 2 on chip), N > 4096
    kRowsPease = 5        // k_pease_rows: Pease's constant-geometry factorisation, one tile per CTA
};

// One compiled single-pass kernel (both directions) for transform length n.
struct RowsVariant {
    int kind;               // RowsKind
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

// One compiled column-transform length for the two passes of Eq. 2.
struct ColsVariant {
    int len;                // column transform length
    int e;                  // complex elements per thread per stage
    int c;                  // columns per CTA
    int tpb;                // threads per CTA
    int nstages;
    int radix[kMaxStages];
    int smem;               // dynamic shared memory, bytes
    const void* k1f;        // pass 1 (column gather + DFT + D^N_M), forward / inverse
    const void* k1i;
    const void* k2f;        // pass 2 (DFT across the columns), forward / inverse
    const void* k2i;
};

const ColsVariant* cols_variant_for_nd(int64_t len, int64_t ncols);  // ND axis passes: wider CTAs where the stride allows
const ColsVariant* cols_variant_for(int64_t len);
const ColsVariant* cols_variants(int* count);
cudaError_t prepare_cols(const ColsVariant& v);
// pass 1: in = x, out = workspace z, post = D^N_M table; pass 2: in = z, out = y.
cudaError_t launch_cols(const ColsVariant& v, int pass, int direction, const float2* in, float2* out,
                        const float2* tw, const float2* post, long long batch, int ncols, cudaStream_t stream);

// D^N_M table in workspace layout: post[k*M + j1] = w_N^(j1*k), k < N/M, j1 < M.
cudaError_t launch_post_twiddles(float2* post, int64_t n, int64_t m, cudaStream_t stream);

// Tensor-core variant (tc.cu): all-radix-16 schedules, DFT_16 as split
// half-precision mma products.  k[prec][dir]: prec 0 = FP16x2, 1 = BF16x2;
// dir 0 = forward, 1 = inverse.
struct TcVariant {
    int n, rows, tpb, nstages, smem;
    const void* k[2][2];
};
const TcVariant* tc_variant_for(int64_t n);
cudaError_t prepare_tc(const TcVariant& v);
// frag: 32 lanes x 32 words; prec as above; sign = exponent sign of the transform.
cudaError_t launch_tc_fragments(uint32_t* frag, int prec, int sign, cudaStream_t s);
// Resident CTAs of the (persistent) tensor-core kernel on the current device.
int tc_grid(const TcVariant& v);
cudaError_t launch_tc(const TcVariant& v, int prec, int direction, const float2* in, float2* out, const float2* tw,
                      const uint32_t* frag, long long batch, int grid_cap, cudaStream_t s);

// Tensor-core variant on tcgen05 / tensor memory (umma.cu): same schedules
// and arithmetic as the mma.sync variant; N = 256 and 4096.
struct UmmaVariant {
    int n, rows, tpb, smem;
    const void* k[2][2];  // [prec][dir]
};
const UmmaVariant* umma_variant_for(int64_t n);
cudaError_t prepare_umma(const UmmaVariant& v);
int umma_grid(const UmmaVariant& v);
// bm: 64 x 32 halves (4 KB) of [Mh; Ml] in the operand layout the kernel expects.
cudaError_t launch_umma_bmat(uint16_t* bm, int prec, int sign, cudaStream_t s);
cudaError_t launch_umma(const UmmaVariant& v, int prec, int direction, const float2* in, float2* out,
                        const float2* tw, const void* bmat, long long batch, int grid_cap, int* status,
                        cudaStream_t s);

// Direct DFT on tcgen05 for small N (direct.cu): y = F_N x as one split
// half-precision matrix product per 128 transforms; N = 8, 16, ..., 64.
struct DirectVariant {
    int n, rows, tpb, smem, bmat_bytes, tmem_cols;
    const void* k[2][2];    // [prec][dir], 16-byte loads
    const void* k32[2][2];  // the same with 32-byte loads, for 32-byte-aligned inputs
};
const DirectVariant* direct_variant_for(int64_t n);
cudaError_t prepare_direct(const DirectVariant& v);
int direct_grid(const DirectVariant& v);
cudaError_t launch_direct_bmat(uint16_t* bm, int n, int prec, int sign, cudaStream_t s);
cudaError_t launch_direct(const DirectVariant& v, int prec, int direction, const float2* in, float2* out,
                          const void* bmat, long long batch, int grid_cap, int* status, cudaStream_t s);

// The direct DFT warp-specialised and pipelined (direct_ws.cu): producers,
// one MMA thread and an epilogue hand tiles over through two tensor-memory slots.
struct DirectWsVariant {
    int n, tpb, smem, tmem_cols;
    const void* k[2][2];  // [prec][dir]
};
const DirectWsVariant* direct_ws_variant_for(int64_t n);
cudaError_t prepare_direct_ws(const DirectWsVariant& v);
int direct_ws_grid(const DirectWsVariant& v);
cudaError_t launch_direct_ws(const DirectWsVariant& v, int prec, int direction, const float2* in, float2* out,
                             const void* bmat, long long batch, int grid_cap, int* status, cudaStream_t s);

// Ragged-batch plans (ragged.cu).
struct RaggedState;
gbfft_status ragged_create(RaggedState** out, const int64_t* n, const int64_t* offsets, int64_t count);
void ragged_destroy(RaggedState* r);
int64_t ragged_total(const RaggedState* r);
gbfft_status ragged_execute(RaggedState* r, int direction, const void* in, void* out, int* status,
                            cudaStream_t s);
gbfft_status ragged_execute_direct(RaggedState* r, int direction, const void* in, void* out, int* status,
                                   cudaStream_t s);
int64_t ragged_num_items(const RaggedState* r);
gbfft_status ragged_set_item_ready(RaggedState* r, int64_t item, int ready);
void ragged_set_wait_ns(RaggedState* r, long long ns);
gbfft_status ragged_autotune(RaggedState* r, int direction, const void* in, void* out, int* status, int reps,
                             float* best_ms);
int ragged_class_split(const RaggedState* r, int64_t n);
int ragged_queue_order(const RaggedState* r);
gbfft_status ragged_set_queue_order(RaggedState* r, int order);
gbfft_status ragged_set_engine(RaggedState* r, int64_t n, int compiled);
int ragged_engine(const RaggedState* r, int64_t n);

// Length table and per-call queues for ragged launches whose transforms change
// from call to call (ragged.cu).
struct RaggedTable;
struct RaggedSpan {
    int64_t n;     // transform length
    long long off; // complex element of the first row in the data buffer
    int64_t rows;  // consecutive rows of length n
    long long dout; // the output rows start dout complex elements after the input rows
};
gbfft_status ragged_table_create(RaggedTable** out);
void ragged_table_destroy(RaggedTable* t);
gbfft_status ragged_table_add(RaggedTable* t, int64_t n, cudaStream_t s, int* cls);
size_t ragged_blob_bytes(int64_t nitems, int64_t nrows);
int64_t ragged_table_build(const RaggedTable* t, const RaggedSpan* spans, int64_t nspans, char* blob, size_t cap,
                           size_t* bytes);
cudaError_t ragged_table_launch(const RaggedTable* t, int direction, float2* data, const char* d_blob,
                                int64_t nitems, int* status, cudaStream_t s);
// Radix schedule the plan uses for length n (stage count; 0 if n is absent).
int ragged_schedule(const RaggedState* r, int64_t n, int* radix);
bool ragged_supported(int64_t n);

// Factorisation-formula front end (formula.cu): whether `text` denotes DFT_n by
// Eq. 2; its DFT leaves in application order, outermost split K (0 if none) and
// whether that split's DFT factors are plain DFT(K), DFT(M) leaves.
bool formula_plan_choice(const char* text, int64_t* n, std::vector<int64_t>* leaves, int64_t* k_top, bool* bare,
                         bool* pease);

// Planner wisdom (autotune.cu): the autotuned choice for (n, dtype, direction).
void wisdom_load_env_once();
bool wisdom_lookup(int64_t n, int dtype, int direction, int* variant, int64_t* k_outer);

// Per-translation-unit variant tables, gathered by the registry in api.cu.
const RowsVariant* rows_variants_pow2(int* count);
const RowsVariant* rows_variants_mixed(int* count);
const RowsVariant* rows_variants_pease(int* count);  // Pease form, N = R^t (pease.cu)
// Complex128 / FP64 single-pass variants (rows_f64.cu).
const RowsVariant* rows_variants_f64(int* count);
int rows_variants_f64_for(int64_t n, const RowsVariant** out, int max_out);

// All variants for length n, in preference order (the first is the default).
int rows_variants_for(int64_t n, const RowsVariant** out, int max_out);
// One-pass cluster variants for 4096 < n <= 32768 (cluster.cu); their radix
// list is the column schedule followed by the cluster size K.
int cluster_variants_for(int64_t n, const RowsVariant** out, int max_out);
bool cluster_is_default(int64_t n);
// The planner's Eq. 2 split N = K * M for the two-pass form (k_req > 0: that K, if valid); false if none.
bool choose_split(int64_t n, int64_t k_req, int64_t* k_out, int64_t* m_out);  // the default plan for n is the cluster kernel (variant 0)
// The one-pass variants of a length: single-CTA rows kernels, else cluster kernels.
int onepass_variants_for(int64_t n, const RowsVariant** out, int max_out);
// Twiddle tables of a cluster variant: the column's stage blocks, then D^N_M.
gbfft_status alloc_cluster_tables(float2** dst, const RowsVariant& v);

// Largest useful grid for a persistent variant on the current device:
// resident CTAs per SM times the SM count (0 on error).
int persistent_grid(const RowsVariant& v);

// Make the variant's kernels accept its dynamic shared memory size.
cudaError_t prepare_rows(const RowsVariant& v);

// Launch a rows variant over `batch` contiguous rows.  `grid_cap` bounds the
// grid of a persistent variant (see persistent_grid); ignored otherwise.
// `status` receives bounded-wait timeouts of the TMA variants (may be null
// for the others).
cudaError_t launch_rows(const RowsVariant& v, int direction, const void* in, void* out, const void* tw,
                        long long batch, int grid_cap, cudaStream_t stream, int* status = nullptr);

// tw[j] = exp(-2*pi*i*j/n) for j < n, evaluated in FP64 on the device.
cudaError_t launch_twiddle_table(float2* tw, int64_t n, cudaStream_t stream);

// Stage twiddle blocks of a schedule (see stockham.cuh): entries and launch.
int stage_twiddle_count(const int* radix, int nstages);
cudaError_t launch_stage_twiddles(float2* tw, int64_t n, const int* radix, int nstages, cudaStream_t stream);
cudaError_t launch_stage_twiddles64(double2* tw, int64_t n, const int* radix, int nstages, cudaStream_t stream);

}  // namespace gbfft
