// The C ABI of include/gbfft.h: plans, execution, variant registry, status.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace gbfft {

int rows_variants_for(int64_t n, const RowsVariant** out, int max_out) {
    int found = 0;
    const RowsVariant* tabs[3];
    int counts[3];
    tabs[0] = rows_variants_pow2(&counts[0]);
    tabs[1] = rows_variants_mixed(&counts[1]);
    tabs[2] = rows_variants_pease(&counts[2]);  // after the Stockham variants: their indices stay put
    for (int t = 0; t < 3; ++t) {
        for (int i = 0; i < counts[t]; ++i) {
            if (tabs[t][i].n == n) {
                if (found < max_out && out) out[found] = &tabs[t][i];
                ++found;
            }
        }
    }
    return found;
}

int onepass_variants_for(int64_t n, const RowsVariant** out, int max_out) {
    const int nr = rows_variants_for(n, out, max_out);
    return nr > 0 ? nr : cluster_variants_for(n, out, max_out);
}

int persistent_grid(const RowsVariant& v) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.kfwd, v.tpb, (size_t)v.smem) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

cudaError_t prepare_rows(const RowsVariant& v) {
    if (v.smem <= 48 * 1024) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(v.kfwd, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(v.kinv, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem);
    return e;
}

cudaError_t launch_rows(const RowsVariant& v, int direction, const void* in, void* out, const void* tw,
                        long long batch, int grid_cap, cudaStream_t stream, int* status) {
    if (batch <= 0) return cudaSuccess;
    long long blocks = (batch + v.rows - 1) / v.rows;
    if ((v.kind == kRowsPersistent || v.kind == kRowsTma) && grid_cap > 0 && blocks > grid_cap) blocks = grid_cap;
    if (v.kind == kRowsCluster) blocks = batch * v.radix[v.nstages - 1];  // one row per cluster of K CTAs
    void* args[] = {(void*)&in, (void*)&out, (void*)&tw, (void*)&batch, (void*)&status};
    const void* fn = direction == GBFFT_FORWARD ? v.kfwd : v.kinv;
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(v.tpb), args, (size_t)v.smem, stream);
}

// Eq. 2 split N = K * M for the two-pass path: M (pass-1 column length) is
// taken from a preference list; K must also be a registered column length.
bool split_ok(int64_t k, int64_t m) {
    // both passes take 16 whole columns per CTA: K (pass 1) and M (pass 2) columns
    return k % 16 == 0 && m % 16 == 0 && cols_variant_for(k) && cols_variant_for(m);
}

bool choose_split(int64_t n, int64_t k_req, int64_t* k_out, int64_t* m_out) {
    if (k_req > 0) {
        if (n % k_req != 0) return false;
        const int64_t m = n / k_req;
        if (!split_ok(k_req, m)) return false;
        *k_out = k_req;
        *m_out = m;
        return true;
    }
    // Inner length M by preference.  From N = 16384 up M = 256 comes first: measured on GB300
    // (2^26 points), N = 16384 / 32768 / 65536 ran at 3436 / 3381 / 3029 GB/s with M = 256
    // against 3356 / 3022 / 2644 with M = 128 (N = 8192 keeps M = 128: 3427 against 3397).
    static const int64_t pref_short[] = {128, 64, 256, 96, 112, 80, 48, 32, 512};
    static const int64_t pref_long[] = {256, 128, 64, 96, 112, 80, 48, 32, 512};
    for (int64_t m : (n >= 16384 ? pref_long : pref_short)) {
        if (n % m == 0 && split_ok(n / m, m)) {
            *k_out = n / m;
            *m_out = m;
            return true;
        }
    }
    return false;
}

}  // namespace gbfft

using namespace gbfft;

enum PlanKind : int { kPlanSingle = 0, kPlanTwoPass = 1, kPlanRagged = 2, kPlanTensorCore = 3, kPlanND = 4 };

struct gbfft_plan_s {
    int64_t n = 0;
    int64_t batch = 0;
    int direction = GBFFT_FORWARD;
    int dtype = GBFFT_C2C_F32;
    int device = 0;
    int kind = kPlanSingle;
    // single pass
    int variant = -1;
    const RowsVariant* rv = nullptr;
    int grid_cap = 0;  // persistent variants: resident CTAs on the device
    float2* tw = nullptr;
    double2* tw64 = nullptr;  // complex128 plans: FP64 stage twiddles
    // two passes (Eq. 2 with N = K * M)
    int64_t k_outer = 1, m_inner = 0;
    const ColsVariant* cv_m = nullptr;  // pass 1: length-M columns
    const ColsVariant* cv_k = nullptr;  // pass 2: length-K columns
    float2* tw_m = nullptr;
    float2* tw_k = nullptr;
    float2* post = nullptr;  // D^N_M in workspace layout
    float2* ws = nullptr;    // workspace z, batch * n complex
    // multi-dimensional (row-major dims[0] x ... x dims[rank-1]): a single-pass row
    // transform along the last axis, then in-place column transforms along the others
    int rank = 1;
    int64_t dims[3] = {0, 0, 0};
    const ColsVariant* cv_nd[2] = {nullptr, nullptr};  // axis rank-2, axis rank-3
    float2* tw_nd[2] = {nullptr, nullptr};
    // ragged batch
    RaggedState* ragged = nullptr;
    // tensor-core split precision (all-radix-16 schedule)
    const TcVariant* tcv = nullptr;
    const UmmaVariant* umv = nullptr;  // tcgen05 engine (variant 1) instead of mma.sync (variant 0)
    const DirectVariant* dv = nullptr;     // direct DFT on tcgen05, one tile at a time per CTA (variant 3)
    const DirectWsVariant* dwv = nullptr;  // the same, warp-specialised and pipelined (variant 2)
    uint16_t* direct_b = nullptr;
    int tc_prec = 0;
    uint32_t* tc_frag = nullptr;
    uint16_t* umma_b = nullptr;
    int* status = nullptr;
    size_t ws_bytes = 0;
    // host-buffer execution: staging ring and its streams/events (created on first use)
    static constexpr int kRing = 3;
    void* stage[kRing] = {nullptr, nullptr, nullptr};
    int64_t stage_rows = 0;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_start = nullptr, ev_in[kRing] = {}, ev_comp[kRing] = {}, ev_out[kRing] = {};
};

namespace {

constexpr int kMaxVariantsPerSize = 16;

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Bytes per complex point of a dtype.
size_t elem_bytes(int dtype) { return dtype == GBFFT_C2C_F64 ? sizeof(double2) : sizeof(float2); }

gbfft_status check_io(const void* in, const void* out, size_t bytes) {
    if (!in || !out) return GBFFT_ERR_INVALID_ARG;
    if (!aligned16(in) || !aligned16(out)) return GBFFT_ERR_ALIGNMENT;
    if (in != out) {
        const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
        if (a < b + bytes && b < a + bytes) return GBFFT_ERR_OVERLAP;
    }
    return GBFFT_OK;
}

void free_plan(gbfft_plan p) {
    if (!p) return;
    if (p->s_in) cudaStreamSynchronize(p->s_in);
    if (p->s_out) cudaStreamSynchronize(p->s_out);
    for (int b = 0; b < gbfft_plan_s::kRing; ++b) {
        if (p->stage[b]) cudaFree(p->stage[b]);
        if (p->ev_in[b]) cudaEventDestroy(p->ev_in[b]);
        if (p->ev_comp[b]) cudaEventDestroy(p->ev_comp[b]);
        if (p->ev_out[b]) cudaEventDestroy(p->ev_out[b]);
    }
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    if (p->ragged) ragged_destroy(p->ragged);
    if (p->tc_frag) cudaFree(p->tc_frag);
    if (p->umma_b) cudaFree(p->umma_b);
    if (p->tw64) cudaFree(p->tw64);
    if (p->direct_b) cudaFree(p->direct_b);
    float2* bufs[] = {p->tw, p->tw_m, p->tw_k, p->post, p->ws, p->tw_nd[0], p->tw_nd[1]};
    for (float2* b : bufs)
        if (b) cudaFree(b);
    if (p->status) cudaFree(p->status);
    delete p;
}

gbfft_status alloc_stage_tables(float2** dst, int64_t n, const int* radix, int nstages) {
    const int cnt = stage_twiddle_count(radix, nstages);
    if (cudaMalloc(dst, sizeof(float2) * (size_t)(cnt > 0 ? cnt : 1)) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return GBFFT_ERR_OOM;
    }
    return launch_stage_twiddles(*dst, n, radix, nstages, 0) == cudaSuccess ? GBFFT_OK : GBFFT_ERR_CUDA;
}

// Direct DFT (variants 2 and 3 of the tensor-core dtypes): one split-precision
// matrix product per 128 transforms, N a multiple of 8 up to 64; `ws` selects
// the warp-specialised, pipelined kernel (variant 2) over the kernel that runs
// each tile's phases one after the other (variant 3).
gbfft_status create_direct(gbfft_plan* out, int64_t n, int64_t batch, int direction, int dtype, bool ws) {
    const DirectVariant* dv = direct_variant_for(n);
    const DirectWsVariant* dwv = ws ? direct_ws_variant_for(n) : nullptr;
    if (!dv || (ws && !dwv)) return GBFFT_ERR_NOT_FOUND;
    // BF16x2 keeps ~16 significand bits: one dense product errs by 4-6e-6 relative
    // L2 at every N, above the 1e-6*log2(N) contract for N <= 64.
    if (dtype == GBFFT_C2C_F32_TC_BF16X2) return GBFFT_ERR_UNSUPPORTED_SIZE;
    gbfft_plan p = new (std::nothrow) gbfft_plan_s();
    if (!p) return GBFFT_ERR_OOM;
    p->kind = kPlanTensorCore;
    p->n = n;
    p->batch = batch;
    p->direction = direction;
    p->dtype = dtype;
    p->dv = dv;
    p->dwv = dwv;
    p->variant = ws ? 2 : 3;
    p->tc_prec = dtype == GBFFT_C2C_F32_TC_FP16X2 ? 0 : 1;
    gbfft_status st = GBFFT_OK;
    if (cudaGetDevice(&p->device) != cudaSuccess || cudaMalloc(&p->status, sizeof(int)) != cudaSuccess ||
        cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&p->direct_b, (size_t)dv->bmat_bytes) != cudaSuccess) {
        cudaGetLastError();
        st = GBFFT_ERR_OOM;
    }
    if (st == GBFFT_OK && (ws ? prepare_direct_ws(*dwv) : prepare_direct(*dv)) != cudaSuccess) st = GBFFT_ERR_CUDA;
    if (st == GBFFT_OK && (p->grid_cap = ws ? direct_ws_grid(*dwv) : direct_grid(*dv)) <= 0) st = GBFFT_ERR_CUDA;
    if (st == GBFFT_OK && launch_direct_bmat(p->direct_b, (int)n, p->tc_prec, direction, 0) != cudaSuccess)
        st = GBFFT_ERR_CUDA;
    if (st == GBFFT_OK && cudaDeviceSynchronize() != cudaSuccess) st = GBFFT_ERR_CUDA;
    if (st != GBFFT_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return GBFFT_OK;
}

gbfft_status create_tc(gbfft_plan* out, int64_t n, int64_t batch, int direction, int dtype, int engine) {
    if (engine == 2 || engine == 3) return create_direct(out, n, batch, direction, dtype, engine == 2);
    const TcVariant* tv = tc_variant_for(n);
    if (!tv) return GBFFT_ERR_UNSUPPORTED_SIZE;
    const UmmaVariant* uv = engine == 1 ? umma_variant_for(n) : nullptr;
    if (engine == 1 && !uv) return GBFFT_ERR_NOT_FOUND;
    // BF16x2 keeps ~17 significand bits; a lone radix-16 stage then errs by ~5e-6
    // relative L2, above the 1e-6*log2(N) = 4e-6 contract at N = 16.
    if (dtype == GBFFT_C2C_F32_TC_BF16X2 && n < 256) return GBFFT_ERR_UNSUPPORTED_SIZE;
    gbfft_plan p = new (std::nothrow) gbfft_plan_s();
    if (!p) return GBFFT_ERR_OOM;
    p->kind = kPlanTensorCore;
    p->n = n;
    p->batch = batch;
    p->direction = direction;
    p->dtype = dtype;
    p->tcv = tv;
    p->umv = uv;
    p->tc_prec = dtype == GBFFT_C2C_F32_TC_FP16X2 ? 0 : 1;
    int radix[kMaxStages];
    for (int s = 0; s < tv->nstages; ++s) radix[s] = 16;
    gbfft_status st = GBFFT_OK;
    if (cudaGetDevice(&p->device) != cudaSuccess || cudaMalloc(&p->status, sizeof(int)) != cudaSuccess ||
        cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess || cudaMalloc(&p->tc_frag, 32 * 32 * 4) != cudaSuccess) {
        cudaGetLastError();
        st = GBFFT_ERR_OOM;
    }
    if (uv) {
        if (st == GBFFT_OK && prepare_umma(*uv) != cudaSuccess) st = GBFFT_ERR_CUDA;
        if (st == GBFFT_OK && (p->grid_cap = umma_grid(*uv)) <= 0) st = GBFFT_ERR_CUDA;
        if (st == GBFFT_OK && cudaMalloc(&p->umma_b, 64 * 32 * 2) != cudaSuccess) {
            cudaGetLastError();
            st = GBFFT_ERR_OOM;
        }
        if (st == GBFFT_OK && launch_umma_bmat(p->umma_b, p->tc_prec, direction, 0) != cudaSuccess) st = GBFFT_ERR_CUDA;
    } else {
        if (st == GBFFT_OK && prepare_tc(*tv) != cudaSuccess) st = GBFFT_ERR_CUDA;
        if (st == GBFFT_OK && (p->grid_cap = tc_grid(*tv)) <= 0) st = GBFFT_ERR_CUDA;
    }
    if (st == GBFFT_OK) st = alloc_stage_tables(&p->tw, n, radix, tv->nstages);
    if (st == GBFFT_OK && launch_tc_fragments(p->tc_frag, p->tc_prec, direction, 0) != cudaSuccess)
        st = GBFFT_ERR_CUDA;
    if (st == GBFFT_OK && cudaDeviceSynchronize() != cudaSuccess) st = GBFFT_ERR_CUDA;
    if (st != GBFFT_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return GBFFT_OK;
}

// Complex128 plan: one single-pass FP64 variant (no two-pass or tensor-core form).
gbfft_status create_f64(gbfft_plan* out, int64_t n, int64_t batch, int direction, int variant, int64_t k_outer) {
    if (k_outer > 0) return GBFFT_ERR_INVALID_ARG;
    const RowsVariant* cands[kMaxVariantsPerSize];
    const int nc = rows_variants_f64_for(n, cands, kMaxVariantsPerSize);
    if (nc == 0) return GBFFT_ERR_UNSUPPORTED_SIZE;
    if (variant < 0) variant = 0;
    if (variant >= nc) return GBFFT_ERR_NOT_FOUND;
    gbfft_plan p = new (std::nothrow) gbfft_plan_s();
    if (!p) return GBFFT_ERR_OOM;
    p->kind = kPlanSingle;
    p->n = n;
    p->batch = batch;
    p->direction = direction;
    p->dtype = GBFFT_C2C_F64;
    p->variant = variant;
    p->rv = cands[variant];
    gbfft_status st = GBFFT_OK;
    const int cnt = stage_twiddle_count(p->rv->radix, p->rv->nstages);
    if (cudaGetDevice(&p->device) != cudaSuccess || cudaMalloc(&p->status, sizeof(int)) != cudaSuccess ||
        cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&p->tw64, sizeof(double2) * (size_t)(cnt > 0 ? cnt : 1)) != cudaSuccess) {
        cudaGetLastError();
        st = GBFFT_ERR_OOM;
    }
    if (st == GBFFT_OK && prepare_rows(*p->rv) != cudaSuccess) st = GBFFT_ERR_CUDA;
    if (st == GBFFT_OK && launch_stage_twiddles64(p->tw64, n, p->rv->radix, p->rv->nstages, 0) != cudaSuccess)
        st = GBFFT_ERR_CUDA;
    if (st == GBFFT_OK && cudaDeviceSynchronize() != cudaSuccess) st = GBFFT_ERR_CUDA;
    if (st != GBFFT_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return GBFFT_OK;
}

gbfft_status create(gbfft_plan* out, int64_t n, int64_t batch, int direction, int dtype, int variant,
                    int64_t k_outer) {
    if (!out) return GBFFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || batch < 0 || k_outer < 0) return GBFFT_ERR_INVALID_ARG;
    if (direction != GBFFT_FORWARD && direction != GBFFT_INVERSE) return GBFFT_ERR_INVALID_ARG;
    if (dtype != GBFFT_C2C_F32 && dtype != GBFFT_C2C_F32_TC_FP16X2 && dtype != GBFFT_C2C_F32_TC_BF16X2 &&
        dtype != GBFFT_C2C_F64)
        return GBFFT_ERR_INVALID_ARG;
    if (variant < 0 && k_outer == 0) {  // no forced choice: use autotuned wisdom when there is some
        wisdom_load_env_once();
        int wv = -1;
        int64_t wk = 0;
        if (wisdom_lookup(n, dtype, direction, &wv, &wk)) {
            if (wk > 0 && dtype == GBFFT_C2C_F32) {
                int64_t kk, mm;
                if (choose_split(n, wk, &kk, &mm)) k_outer = wk;
            } else if (wv >= 0) {
                const int limit = dtype == GBFFT_C2C_F32   ? onepass_variants_for(n, nullptr, 0)
                                  : dtype == GBFFT_C2C_F64 ? rows_variants_f64_for(n, nullptr, 0)
                                                           : 4;
                if (wv < limit) variant = wv;
            }
        }
    }
    if (dtype == GBFFT_C2C_F64) return create_f64(out, n, batch, direction, variant, k_outer);
    if (dtype != GBFFT_C2C_F32) {
        if (k_outer > 0) return GBFFT_ERR_INVALID_ARG;
        if (variant > 3) return GBFFT_ERR_NOT_FOUND;
        // default engine: tcgen05 Stockham where it exists (N = 256, 4096); for FP16x2 the direct
        // DFT where it exists (N = 8 ... 64): pipelined (variant 2; at N = 16 6.28 TB/s against 5.43
        // for the mma.sync Stockham), except at N = 8, where the one-tile-at-a-time kernel
        // (variant 3) measured 3 % faster; else mma.sync Stockham (variant 0)
        const bool fp16_direct = dtype == GBFFT_C2C_F32_TC_FP16X2 && direct_variant_for(n);
        const int engine = variant >= 0         ? variant
                           : umma_variant_for(n) ? 1
                           : fp16_direct         ? (n == 8 ? 3 : 2)
                           : tc_variant_for(n)   ? 0
                           : direct_variant_for(n) ? 2
                                                   : 0;
        return create_tc(out, n, batch, direction, dtype, engine);
    }

    const RowsVariant* cands[kMaxVariantsPerSize];
    const int nc = onepass_variants_for(n, cands, kMaxVariantsPerSize);
    int64_t kk = 0, mm = 0;
    // Above 4096 the default is Eq. 2 as two passes, except at the lengths where the one-pass
    // cluster kernel (the row kept on chip, exchanged through distributed shared memory) measured
    // faster on GB300 (cluster_is_default); elsewhere the cluster kernels run when forced, when
    // the autotuner picks them, or when no split exists.
    const bool cluster_only = nc > 0 && rows_variants_for(n, nullptr, 0) == 0;
    const bool two_pass =
        k_outer > 0 ||
        (variant < 0 && (nc == 0 || (cluster_only && !cluster_is_default(n) && choose_split(n, 0, &kk, &mm))));
    if (two_pass) {
        if (!choose_split(n, k_outer, &kk, &mm)) return k_outer > 0 ? GBFFT_ERR_NOT_FOUND : GBFFT_ERR_UNSUPPORTED_SIZE;
    } else {
        if (nc == 0) return GBFFT_ERR_UNSUPPORTED_SIZE;
        if (variant < 0) variant = 0;
        if (variant >= nc) return GBFFT_ERR_NOT_FOUND;
    }

    gbfft_plan p = new (std::nothrow) gbfft_plan_s();
    if (!p) return GBFFT_ERR_OOM;
    p->n = n;
    p->batch = batch;
    p->direction = direction;
    p->dtype = dtype;
    if (cudaGetDevice(&p->device) != cudaSuccess || cudaMalloc(&p->status, sizeof(int)) != cudaSuccess ||
        cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        free_plan(p);
        return GBFFT_ERR_CUDA;
    }
    gbfft_status st = GBFFT_OK;
    if (two_pass) {
        p->kind = kPlanTwoPass;
        p->k_outer = kk;
        p->m_inner = mm;
        p->cv_m = cols_variant_for(mm);
        p->cv_k = cols_variant_for(kk);
        p->ws_bytes = sizeof(float2) * (size_t)n * (size_t)batch;
        if (prepare_cols(*p->cv_m) != cudaSuccess || prepare_cols(*p->cv_k) != cudaSuccess) st = GBFFT_ERR_CUDA;
        if (st == GBFFT_OK) st = alloc_stage_tables(&p->tw_m, mm, p->cv_m->radix, p->cv_m->nstages);
        if (st == GBFFT_OK) st = alloc_stage_tables(&p->tw_k, kk, p->cv_k->radix, p->cv_k->nstages);
        if (st == GBFFT_OK) {
            if (cudaMalloc(&p->post, sizeof(float2) * (size_t)n) != cudaSuccess ||
                (p->ws_bytes && cudaMalloc(&p->ws, p->ws_bytes) != cudaSuccess)) {
                cudaGetLastError();
                st = GBFFT_ERR_OOM;
            }
        }
        if (st == GBFFT_OK && launch_post_twiddles(p->post, n, mm, 0) != cudaSuccess) st = GBFFT_ERR_CUDA;
    } else {
        p->kind = kPlanSingle;
        p->variant = variant;
        p->rv = cands[variant];
        if (prepare_rows(*p->rv) != cudaSuccess) st = GBFFT_ERR_CUDA;
        if (st == GBFFT_OK && (p->rv->kind == kRowsPersistent || p->rv->kind == kRowsTma)) {
            p->grid_cap = persistent_grid(*p->rv);
            if (p->grid_cap <= 0) st = GBFFT_ERR_CUDA;
        }
        if (st == GBFFT_OK)
            st = p->rv->kind == kRowsCluster ? alloc_cluster_tables(&p->tw, *p->rv)
                                             : alloc_stage_tables(&p->tw, n, p->rv->radix, p->rv->nstages);
    }
    // Tables are built on the legacy stream and complete before the plan is returned.
    if (st == GBFFT_OK && cudaDeviceSynchronize() != cudaSuccess) st = GBFFT_ERR_CUDA;
    if (st != GBFFT_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return GBFFT_OK;
}

// Enqueue the transform of `rows` rows from `in` to `out` (device pointers).
cudaError_t run_device(gbfft_plan p, const void* vin, void* vout, int64_t rows, cudaStream_t s) {
    if (p->dtype == GBFFT_C2C_F64)
        return launch_rows(*p->rv, p->direction, vin, vout, p->tw64, (long long)rows, 0, s, p->status);
    const float2* in = (const float2*)vin;
    float2* out = (float2*)vout;
    if (p->kind == kPlanTensorCore && p->dwv)
        return launch_direct_ws(*p->dwv, p->tc_prec, p->direction, in, out, p->direct_b, (long long)rows, p->grid_cap,
                                p->status, s);
    if (p->kind == kPlanTensorCore && p->dv)
        return launch_direct(*p->dv, p->tc_prec, p->direction, in, out, p->direct_b, (long long)rows, p->grid_cap,
                             p->status, s);
    if (p->kind == kPlanTensorCore && p->umv)
        return launch_umma(*p->umv, p->tc_prec, p->direction, in, out, p->tw, p->umma_b, (long long)rows,
                           p->grid_cap, p->status, s);
    if (p->kind == kPlanTensorCore)
        return launch_tc(*p->tcv, p->tc_prec, p->direction, in, out, p->tw, p->tc_frag, (long long)rows,
                         p->grid_cap, s);
    if (p->kind == kPlanSingle)
        return launch_rows(*p->rv, p->direction, in, out, p->tw, (long long)rows, p->grid_cap, s, p->status);
    if (p->kind == kPlanND) {
        // axis rank-1: rows of length dims[rank-1]; then each other axis as columns, in place
        const int64_t last = p->dims[p->rank - 1];
        const int64_t per = p->n / last;  // rows per array
        cudaError_t e = launch_rows(*p->rv, p->direction, in, out, p->tw, (long long)(rows * per), p->grid_cap, s,
                                    p->status);
        int64_t inner = last;             // elements after the axis being transformed
        for (int ax = p->rank - 2, c = 0; e == cudaSuccess && ax >= 0; --ax, ++c) {
            const int64_t outer = p->n / (p->dims[ax] * inner);  // arrays of (dims[ax] x inner) per item
            e = launch_cols(*p->cv_nd[c], 2, p->direction, out, out, p->tw_nd[c], nullptr,
                            (long long)(rows * outer), (int)inner, s);
            inner *= p->dims[ax];
        }
        return e;
    }
    cudaError_t e = launch_cols(*p->cv_m, 1, p->direction, in, p->ws, p->tw_m, p->post, (long long)rows,
                                (int)p->k_outer, s);
    if (e != cudaSuccess) return e;
    return launch_cols(*p->cv_k, 2, p->direction, p->ws, out, p->tw_k, nullptr, (long long)rows,
                       (int)p->m_inner, s);
}

}  // namespace

extern "C" {

const char* gbfft_status_string(gbfft_status s) {
    switch (s) {
        case GBFFT_OK: return "ok";
        case GBFFT_ERR_INVALID_ARG: return "invalid argument";
        case GBFFT_ERR_UNSUPPORTED_SIZE: return "unsupported transform size";
        case GBFFT_ERR_ALIGNMENT: return "pointer not 16-byte aligned";
        case GBFFT_ERR_OVERLAP: return "input and output partially overlap";
        case GBFFT_ERR_OOM: return "device out of memory";
        case GBFFT_ERR_BUDGET: return "memory budget exceeded";
        case GBFFT_ERR_CUDA: return "CUDA error";
        case GBFFT_ERR_TIMEOUT: return "bounded wait timed out";
        case GBFFT_ERR_DEVICE_STATUS: return "device kernel reported an error";
        case GBFFT_ERR_NOT_FOUND: return "not found";
    }
    return "unknown status";
}

int gbfft_version(void) { return 100; }

gbfft_status gbfft_plan_create(gbfft_plan* out, int64_t n, int64_t batch, int direction, int dtype) {
    return create(out, n, batch, direction, dtype, -1, 0);
}

gbfft_status gbfft_plan_create_variant(gbfft_plan* out, int64_t n, int64_t batch, int direction, int dtype,
                                       int variant) {
    if (variant < 0) return GBFFT_ERR_NOT_FOUND;
    return create(out, n, batch, direction, dtype, variant, 0);
}

gbfft_status gbfft_plan_create_twopass(gbfft_plan* out, int64_t n, int64_t batch, int direction, int dtype,
                                       int64_t k_outer) {
    if (k_outer < 0) return GBFFT_ERR_INVALID_ARG;
    if (k_outer == 0) {
        int64_t kk, mm;
        if (out) *out = nullptr;
        if (n < 1) return GBFFT_ERR_INVALID_ARG;
        if (!choose_split(n, 0, &kk, &mm)) return GBFFT_ERR_UNSUPPORTED_SIZE;
        k_outer = kk;
    }
    return create(out, n, batch, direction, dtype, -1, k_outer);
}

// Multi-dimensional plan: DFT_{d0} (x) ... (x) DFT_{d(r-1)} on row-major arrays
// (the Kronecker product of Table I applied to whole transforms): the last
// axis by a single-pass row kernel, every other axis by the column kernel of
// Eq. 2's second pass (length-d transforms down `inner` columns, in place).
gbfft_status gbfft_plan_create_nd(gbfft_plan* out, int rank, const int64_t* dims, int64_t batch, int direction,
                                  int dtype) {
    if (!out) return GBFFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (rank < 1 || rank > 3 || !dims || batch < 0) return GBFFT_ERR_INVALID_ARG;
    if (direction != GBFFT_FORWARD && direction != GBFFT_INVERSE) return GBFFT_ERR_INVALID_ARG;
    if (dtype != GBFFT_C2C_F32) return GBFFT_ERR_INVALID_ARG;
    for (int i = 0; i < rank; ++i)
        if (dims[i] < 1 || dims[i] > ((int64_t)1 << 20)) return GBFFT_ERR_INVALID_ARG;
    if (rank == 1) return create(out, dims[0], batch, direction, dtype, -1, 0);
    const int64_t last = dims[rank - 1];
    const RowsVariant* cands[kMaxVariantsPerSize];
    if (rows_variants_for(last, cands, kMaxVariantsPerSize) == 0) return GBFFT_ERR_UNSUPPORTED_SIZE;
    if (last % 16 != 0) return GBFFT_ERR_UNSUPPORTED_SIZE;  // column kernels take 16 columns per CTA
    const ColsVariant* cv[2] = {nullptr, nullptr};
    int64_t stride = last;  // columns of the axis pass = product of the later dimensions
    for (int ax = rank - 2, c = 0; ax >= 0; --ax, ++c) {
        cv[c] = cols_variant_for_nd(dims[ax], stride);
        if (!cv[c]) return GBFFT_ERR_UNSUPPORTED_SIZE;
        stride *= dims[ax];
    }
    int64_t total = 1;
    for (int i = 0; i < rank; ++i) total *= dims[i];
    if (total > ((int64_t)1 << 31)) return GBFFT_ERR_INVALID_ARG;
    gbfft_plan p = new (std::nothrow) gbfft_plan_s();
    if (!p) return GBFFT_ERR_OOM;
    p->kind = kPlanND;
    p->rank = rank;
    for (int i = 0; i < rank; ++i) p->dims[i] = dims[i];
    p->n = total;
    p->batch = batch;
    p->direction = direction;
    p->dtype = dtype;
    p->variant = 0;
    p->rv = cands[0];
    gbfft_status st = GBFFT_OK;
    if (cudaGetDevice(&p->device) != cudaSuccess || cudaMalloc(&p->status, sizeof(int)) != cudaSuccess ||
        cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        st = GBFFT_ERR_CUDA;
    }
    if (st == GBFFT_OK && prepare_rows(*p->rv) != cudaSuccess) st = GBFFT_ERR_CUDA;
    if (st == GBFFT_OK && (p->rv->kind == kRowsPersistent || p->rv->kind == kRowsTma)) {
        p->grid_cap = persistent_grid(*p->rv);
        if (p->grid_cap <= 0) st = GBFFT_ERR_CUDA;
    }
    if (st == GBFFT_OK) st = alloc_stage_tables(&p->tw, last, p->rv->radix, p->rv->nstages);
    for (int c = 0; st == GBFFT_OK && c < rank - 1; ++c) {
        p->cv_nd[c] = cv[c];
        if (prepare_cols(*cv[c]) != cudaSuccess) st = GBFFT_ERR_CUDA;
        if (st == GBFFT_OK) st = alloc_stage_tables(&p->tw_nd[c], cv[c]->len, cv[c]->radix, cv[c]->nstages);
    }
    if (st == GBFFT_OK && cudaDeviceSynchronize() != cudaSuccess) st = GBFFT_ERR_CUDA;
    if (st != GBFFT_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return GBFFT_OK;
}

gbfft_status gbfft_plan_dims(gbfft_plan p, int* rank, int64_t* dims) {
    if (!p) return GBFFT_ERR_INVALID_ARG;
    const int r = p->kind == kPlanND ? p->rank : 1;
    if (rank) *rank = r;
    if (dims)
        for (int i = 0; i < r; ++i) dims[i] = p->kind == kPlanND ? p->dims[i] : p->n;
    return GBFFT_OK;
}

// A plan that follows a factorisation formula as literally as the compiled
// kernels allow; *match: 2 = the formula's own schedule (single pass with its
// radix sequence, or Eq. 2's two passes with its outermost split over plain
// DFT factors), 1 = the same radices in another stage order or the outermost
// split with the inner factors on the column kernels' own schedules, 0 = the
// default plan for N (the formula still denotes DFT_N).
gbfft_status gbfft_plan_create_formula(gbfft_plan* out, const char* formula, int64_t batch, int direction, int dtype,
                                       int* match) {
    if (out) *out = nullptr;
    if (match) *match = 0;
    if (!out) return GBFFT_ERR_INVALID_ARG;
    int64_t n = 0, k_top = 0;
    std::vector<int64_t> leaves;
    bool bare = false, pease = false;
    if (!formula_plan_choice(formula, &n, &leaves, &k_top, &bare, &pease)) return GBFFT_ERR_INVALID_ARG;
    int exact = -1, multi = -1;
    if (dtype == GBFFT_C2C_F32 || dtype == GBFFT_C2C_F64) {
        const RowsVariant* cands[kMaxVariantsPerSize];
        const int nc = dtype == GBFFT_C2C_F32 ? onepass_variants_for(n, cands, kMaxVariantsPerSize)
                                              : rows_variants_f64_for(n, cands, kMaxVariantsPerSize);
        std::vector<int64_t> want = leaves;
        std::sort(want.begin(), want.end());
        for (int v = 0; v < nc && v < kMaxVariantsPerSize; ++v) {
            // the same factorisation: a Pease formula runs the Pease kernel, any other the Stockham stages
            const bool same_form = (cands[v]->kind == kRowsPease) == pease;
            std::vector<int64_t> have(cands[v]->radix, cands[v]->radix + cands[v]->nstages);
            if (exact < 0 && same_form && have == leaves) exact = v;
            std::sort(have.begin(), have.end());
            if (multi < 0 && cands[v]->kind != kRowsPease && have == want) multi = v;
        }
    }
    int64_t kk = 0, mm = 0;
    const bool split_ok = dtype == GBFFT_C2C_F32 && k_top > 0 && choose_split(n, k_top, &kk, &mm);
    gbfft_status st;
    int m = 0;
    if (exact >= 0) {
        st = create(out, n, batch, direction, dtype, exact, 0);
        m = 2;
    } else if (split_ok && bare) {
        st = create(out, n, batch, direction, dtype, -1, k_top);
        m = 2;
    } else if (multi >= 0) {
        st = create(out, n, batch, direction, dtype, multi, 0);
        m = 1;
    } else if (split_ok) {
        st = create(out, n, batch, direction, dtype, -1, k_top);
        m = 1;
    } else {
        st = create(out, n, batch, direction, dtype, -1, 0);
    }
    if (st == GBFFT_OK && match) *match = m;
    return st;
}

gbfft_status gbfft_execute(gbfft_plan p, const void* in, void* out, void* cuda_stream) {
    if (!p || p->kind == kPlanRagged) return GBFFT_ERR_INVALID_ARG;
    if (p->batch == 0) return GBFFT_OK;
    const size_t bytes = elem_bytes(p->dtype) * (size_t)p->n * (size_t)p->batch;
    gbfft_status st = check_io(in, out, bytes);
    if (st != GBFFT_OK) return st;
    cudaError_t e = run_device(p, in, out, p->batch, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) cudaGetLastError();  // a failed launch must not surface in later calls
    return e == cudaSuccess ? GBFFT_OK : GBFFT_ERR_CUDA;
}

// Chunked host -> device -> host pipeline over a ring of staging buffers:
// while chunk c is transformed on the caller's stream, chunk c+1 is being
// copied in and chunk c-1 copied out on two internal streams.  Buffers the
// device can address directly skip the ring (see device_address).

// The address at which the device reaches `p` (device or managed memory, or
// page-locked host memory mapped into the device's address space), or null.
static const void* device_address(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged || a.type == cudaMemoryTypeHost)
        return a.devicePointer;
    return nullptr;
}

gbfft_status gbfft_execute_host(gbfft_plan p, const void* host_in, void* host_out, void* cuda_stream) {
    if (!p || !host_in || !host_out || p->kind == kPlanRagged) return GBFFT_ERR_INVALID_ARG;
    if (p->batch == 0) return GBFFT_OK;
    const size_t row_bytes = elem_bytes(p->dtype) * (size_t)p->n;
    const size_t bytes = row_bytes * (size_t)p->batch;
    if (host_in != host_out) {
        const uintptr_t a = (uintptr_t)host_in, b = (uintptr_t)host_out;
        if (a < b + bytes && b < a + bytes) return GBFFT_ERR_OVERLAP;
    }
    // Buffers the device can address (page-locked host memory mapped into its address space - reached
    // over NVLink-C2C on a Grace-Blackwell node - or device memory): the plan's kernels read and write
    // them directly, with no staging copies.
    {
        const void* din = device_address(host_in);
        void* dout = const_cast<void*>(device_address(host_out));
        if (din && dout && ((uintptr_t)din & 15u) == 0 && ((uintptr_t)dout & 15u) == 0)
            return run_device(p, din, dout, p->batch, (cudaStream_t)cuda_stream) == cudaSuccess ? GBFFT_OK
                                                                                              : GBFFT_ERR_CUDA;
    }
    constexpr size_t kChunkBytes = size_t(32) << 20;
    if (!p->stage[0]) {
        int64_t rows = (int64_t)(kChunkBytes / row_bytes);
        if (rows < 1) rows = 1;
        if (rows > p->batch) rows = p->batch;
        p->stage_rows = rows;
        for (int b = 0; b < gbfft_plan_s::kRing; ++b) {
            if (cudaMalloc(&p->stage[b], row_bytes * (size_t)rows) != cudaSuccess) {
                cudaGetLastError();
                for (int c = 0; c <= b; ++c) {
                    if (p->stage[c]) cudaFree(p->stage[c]);
                    p->stage[c] = nullptr;
                }
                return GBFFT_ERR_OOM;
            }
        }
        if (cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming) != cudaSuccess)
            return GBFFT_ERR_CUDA;
        for (int b = 0; b < gbfft_plan_s::kRing; ++b)
            if (cudaEventCreateWithFlags(&p->ev_in[b], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&p->ev_comp[b], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&p->ev_out[b], cudaEventDisableTiming) != cudaSuccess)
                return GBFFT_ERR_CUDA;
    }
    cudaStream_t su = (cudaStream_t)cuda_stream;
    const char* hin = (const char*)host_in;
    char* hout = (char*)host_out;
    bool ok = cudaEventRecord(p->ev_start, su) == cudaSuccess &&
              cudaStreamWaitEvent(p->s_in, p->ev_start, 0) == cudaSuccess;
    int used = 0;
    for (int64_t r0 = 0, c = 0; ok && r0 < p->batch; r0 += p->stage_rows, ++c) {
        const int b = (int)(c % gbfft_plan_s::kRing);
        const int64_t rows = (p->batch - r0) < p->stage_rows ? (p->batch - r0) : p->stage_rows;
        const size_t off = (size_t)r0 * row_bytes, nb = (size_t)rows * row_bytes;
        if (c >= gbfft_plan_s::kRing) ok = ok && cudaStreamWaitEvent(p->s_in, p->ev_out[b], 0) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(p->stage[b], hin + off, nb, cudaMemcpyHostToDevice, p->s_in) == cudaSuccess;
        ok = ok && cudaEventRecord(p->ev_in[b], p->s_in) == cudaSuccess;
        ok = ok && cudaStreamWaitEvent(su, p->ev_in[b], 0) == cudaSuccess;
        ok = ok && run_device(p, p->stage[b], p->stage[b], rows, su) == cudaSuccess;
        ok = ok && cudaEventRecord(p->ev_comp[b], su) == cudaSuccess;
        ok = ok && cudaStreamWaitEvent(p->s_out, p->ev_comp[b], 0) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(hout + off, p->stage[b], nb, cudaMemcpyDeviceToHost, p->s_out) == cudaSuccess;
        ok = ok && cudaEventRecord(p->ev_out[b], p->s_out) == cudaSuccess;
        if (used < gbfft_plan_s::kRing) ++used;
    }
    for (int b = 0; ok && b < used; ++b) ok = cudaStreamWaitEvent(su, p->ev_out[b], 0) == cudaSuccess;
    if (!ok) cudaGetLastError();
    return ok ? GBFFT_OK : GBFFT_ERR_CUDA;
}

gbfft_status gbfft_destroy(gbfft_plan p) {
    free_plan(p);
    return GBFFT_OK;
}

gbfft_status gbfft_plan_info(gbfft_plan p, int64_t* n, int64_t* batch, int* direction, int* nstages,
                             int* radices, int* variant, size_t* workspace_bytes) {
    if (!p) return GBFFT_ERR_INVALID_ARG;
    if (n) *n = p->n;
    if (batch) *batch = p->batch;
    if (direction) *direction = p->direction;
    int ns = 0;
    int rad[2 * kMaxStages];
    if (p->kind == kPlanRagged) {
        // no single schedule: one per length class
    } else if (p->kind == kPlanTensorCore && p->dv) {
        rad[ns++] = (int)p->n;  // the direct DFT: one dense stage of radix N
    } else if (p->kind == kPlanTensorCore) {
        for (int i = 0; i < p->tcv->nstages; ++i) rad[ns++] = 16;
    } else if (p->kind == kPlanSingle || p->kind == kPlanND) {  // ND: the last axis' row schedule
        for (int i = 0; i < p->rv->nstages; ++i) rad[ns++] = p->rv->radix[i];
    } else {
        for (int i = 0; i < p->cv_m->nstages; ++i) rad[ns++] = p->cv_m->radix[i];
        for (int i = 0; i < p->cv_k->nstages; ++i) rad[ns++] = p->cv_k->radix[i];
    }
    if (nstages) *nstages = ns < kMaxStages ? ns : kMaxStages;
    if (radices)
        for (int i = 0; i < ns && i < kMaxStages; ++i) radices[i] = rad[i];
    if (variant) *variant = p->kind == kPlanSingle ? p->variant : (p->kind == kPlanTensorCore ? (p->dwv ? 2 : (p->dv ? 3 : (p->umv ? 1 : 0))) : -1);
    if (workspace_bytes) *workspace_bytes = p->ws_bytes;
    return GBFFT_OK;
}

gbfft_status gbfft_plan_factors(gbfft_plan p, int64_t* k_outer, int64_t* m_inner) {
    if (!p || p->kind == kPlanRagged) return GBFFT_ERR_INVALID_ARG;
    const bool one = p->kind != kPlanTwoPass;
    if (k_outer) *k_outer = one ? 1 : p->k_outer;
    if (m_inner) *m_inner = one ? p->n : p->m_inner;
    return GBFFT_OK;
}

gbfft_status gbfft_plan_ragged(gbfft_plan* out, const int64_t* n, const int64_t* offsets, int64_t count,
                               int direction, int dtype) {
    if (!out) return GBFFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (direction != GBFFT_FORWARD && direction != GBFFT_INVERSE) return GBFFT_ERR_INVALID_ARG;
    if (dtype != GBFFT_C2C_F32 || !n || !offsets || count < 1) return GBFFT_ERR_INVALID_ARG;
    for (int64_t i = 0; i < count; ++i) {
        if (n[i] < 1 || offsets[i] < 0) return GBFFT_ERR_INVALID_ARG;
        if (!ragged_supported(n[i])) return GBFFT_ERR_UNSUPPORTED_SIZE;
    }
    gbfft_plan p = new (std::nothrow) gbfft_plan_s();
    if (!p) return GBFFT_ERR_OOM;
    p->kind = kPlanRagged;
    p->direction = direction;
    p->dtype = dtype;
    p->batch = count;
    if (cudaGetDevice(&p->device) != cudaSuccess || cudaMalloc(&p->status, sizeof(int)) != cudaSuccess ||
        cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        free_plan(p);
        return GBFFT_ERR_CUDA;
    }
    gbfft_status st = ragged_create(&p->ragged, n, offsets, count);
    if (st != GBFFT_OK) {
        free_plan(p);
        return st;
    }
    p->n = ragged_total(p->ragged);
    *out = p;
    return GBFFT_OK;
}

gbfft_status gbfft_execute_ragged(gbfft_plan p, const void* in, void* out, void* cuda_stream) {
    if (!p || p->kind != kPlanRagged) return GBFFT_ERR_INVALID_ARG;
    gbfft_status st = check_io(in, out, sizeof(float2) * (size_t)ragged_total(p->ragged));
    if (st != GBFFT_OK) return st;
    return ragged_execute(p->ragged, p->direction, in, out, p->status, (cudaStream_t)cuda_stream);
}

gbfft_status gbfft_ragged_autotune(gbfft_plan p, const void* in, void* out, int reps, float* best_ms) {
    if (!p || p->kind != kPlanRagged) return GBFFT_ERR_INVALID_ARG;
    gbfft_status st = check_io(in, out, sizeof(float2) * (size_t)ragged_total(p->ragged));
    if (st != GBFFT_OK) return st;
    return ragged_autotune(p->ragged, p->direction, in, out, p->status, reps, best_ms);
}

int64_t gbfft_ragged_num_items(gbfft_plan p) {
    if (!p || p->kind != kPlanRagged) return -1;
    return ragged_num_items(p->ragged);
}

gbfft_status gbfft_ragged_set_item_ready(gbfft_plan p, int64_t item, int ready) {
    if (!p || p->kind != kPlanRagged) return GBFFT_ERR_INVALID_ARG;
    return ragged_set_item_ready(p->ragged, item, ready);
}

gbfft_status gbfft_ragged_set_wait_limit(gbfft_plan p, int64_t nanoseconds) {
    if (!p || p->kind != kPlanRagged || nanoseconds < 1000 || nanoseconds > 10000000000LL)
        return GBFFT_ERR_INVALID_ARG;
    ragged_set_wait_ns(p->ragged, (long long)nanoseconds);
    return GBFFT_OK;
}

gbfft_status gbfft_ragged_set_queue_order(gbfft_plan p, int order) {
    if (!p || p->kind != kPlanRagged || order < 0 || order > 2) return GBFFT_ERR_INVALID_ARG;
    return ragged_set_queue_order(p->ragged, order);
}

int gbfft_ragged_queue_order(gbfft_plan p) {
    if (!p || p->kind != kPlanRagged) return -1;
    return ragged_queue_order(p->ragged);
}

int gbfft_ragged_schedule(gbfft_plan p, int64_t n, int* radices) {
    if (!p || p->kind != kPlanRagged) return -1;
    int rad[kMaxStages];
    const int ns = ragged_schedule(p->ragged, n, rad);
    if (radices)
        for (int i = 0; i < ns; ++i) radices[i] = rad[i];
    return ns;
}

gbfft_status gbfft_ragged_set_engine(gbfft_plan p, int64_t n, int compiled) {
    if (!p || p->kind != kPlanRagged || n < 0 || (compiled != 0 && compiled != 1)) return GBFFT_ERR_INVALID_ARG;
    return ragged_set_engine(p->ragged, n, compiled);
}

int gbfft_ragged_engine(gbfft_plan p, int64_t n) {
    if (!p || p->kind != kPlanRagged) return -1;
    return ragged_engine(p->ragged, n);
}

int gbfft_ragged_tile_split(gbfft_plan p, int64_t n) {
    if (!p || p->kind != kPlanRagged) return 0;
    return ragged_class_split(p->ragged, n);
}

int gbfft_num_variants(int64_t n) { return onepass_variants_for(n, nullptr, 0); }

gbfft_status gbfft_variant_info(int64_t n, int index, int* nstages, int* radices, int* rows_per_cta,
                                int* threads_per_cta, int* smem_bytes) {
    const RowsVariant* cands[kMaxVariantsPerSize];
    const int nc = onepass_variants_for(n, cands, kMaxVariantsPerSize);
    if (index < 0 || index >= nc) return GBFFT_ERR_NOT_FOUND;
    const RowsVariant* v = cands[index];
    if (nstages) *nstages = v->nstages;
    if (radices)
        for (int i = 0; i < v->nstages; ++i) radices[i] = v->radix[i];
    if (rows_per_cta) *rows_per_cta = v->rows;
    if (threads_per_cta) *threads_per_cta = v->tpb;
    if (smem_bytes) *smem_bytes = v->smem;
    return GBFFT_OK;
}

int gbfft_plan_grid_cap(gbfft_plan p) { return p ? p->grid_cap : -1; }

int gbfft_variant_kind(int64_t n, int index) {
    const RowsVariant* cands[kMaxVariantsPerSize];
    const int nc = onepass_variants_for(n, cands, kMaxVariantsPerSize);
    if (index < 0 || index >= nc) return -1;
    return cands[index]->kind;
}

gbfft_status gbfft_plan_device_status(gbfft_plan p) {
    if (!p) return GBFFT_ERR_INVALID_ARG;
    int h = 0;
    if (cudaMemcpy(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GBFFT_ERR_CUDA;
    if (h != 0) {
        cudaMemset(p->status, 0, sizeof(int));
        return h == GBFFT_ERR_TIMEOUT ? GBFFT_ERR_TIMEOUT : GBFFT_ERR_DEVICE_STATUS;
    }
    return GBFFT_OK;
}

}  // extern "C"
