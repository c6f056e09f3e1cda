// The C ABI of include/gbfft.h: plans, execution, variant registry, status.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"

namespace gbfft {

int rows_variants_for(int64_t n, const RowsVariant** out, int max_out) {
    int found = 0;
    int cnt = 0;
    const RowsVariant* tabs[2];
    int counts[2];
    tabs[0] = rows_variants_pow2(&counts[0]);
    tabs[1] = rows_variants_mixed(&counts[1]);
    for (int t = 0; t < 2; ++t) {
        for (int i = 0; i < counts[t]; ++i) {
            if (tabs[t][i].n == n) {
                if (found < max_out && out) out[found] = &tabs[t][i];
                ++found;
            }
        }
    }
    (void)cnt;
    return found;
}

cudaError_t launch_rows(const RowsVariant& v, int direction, const float2* in, float2* out, const float2* tw,
                        long long batch, cudaStream_t stream) {
    if (batch <= 0) return cudaSuccess;
    const long long blocks = (batch + v.rows - 1) / v.rows;
    void* args[] = {(void*)&in, (void*)&out, (void*)&tw, (void*)&batch};
    const void* fn = direction == GBFFT_FORWARD ? v.kfwd : v.kinv;
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(v.tpb), args, (size_t)v.smem, stream);
}

}  // namespace gbfft

using namespace gbfft;

struct gbfft_plan_s {
    int64_t n = 0;
    int64_t batch = 0;
    int direction = GBFFT_FORWARD;
    int dtype = GBFFT_C2C_F32;
    int device = 0;
    int variant = -1;
    const RowsVariant* rv = nullptr;
    float2* tw = nullptr;
    int* status = nullptr;
    size_t ws_bytes = 0;
    // host-buffer execution: staging ring and its streams/events (created on first use)
    static constexpr int kRing = 3;
    float2* stage[kRing] = {nullptr, nullptr, nullptr};
    int64_t stage_rows = 0;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_start = nullptr, ev_in[kRing] = {}, ev_comp[kRing] = {}, ev_out[kRing] = {};
};

namespace {

constexpr int kMaxVariantsPerSize = 16;

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

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
    if (p->tw) cudaFree(p->tw);
    if (p->status) cudaFree(p->status);
    delete p;
}

gbfft_status create(gbfft_plan* out, int64_t n, int64_t batch, int direction, int dtype, int variant) {
    if (!out) return GBFFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || batch < 0) return GBFFT_ERR_INVALID_ARG;
    if (direction != GBFFT_FORWARD && direction != GBFFT_INVERSE) return GBFFT_ERR_INVALID_ARG;
    if (dtype != GBFFT_C2C_F32) return GBFFT_ERR_INVALID_ARG;

    const RowsVariant* cands[kMaxVariantsPerSize];
    const int nc = rows_variants_for(n, cands, kMaxVariantsPerSize);
    if (nc == 0) return GBFFT_ERR_UNSUPPORTED_SIZE;
    if (variant < 0) variant = 0;
    if (variant >= nc) return GBFFT_ERR_NOT_FOUND;

    gbfft_plan p = new (std::nothrow) gbfft_plan_s();
    if (!p) return GBFFT_ERR_OOM;
    p->n = n;
    p->batch = batch;
    p->direction = direction;
    p->dtype = dtype;
    p->variant = variant;
    p->rv = cands[variant];
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return GBFFT_ERR_CUDA;
    }
    if (cudaMalloc(&p->tw, sizeof(float2) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&p->status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        free_plan(p);
        return GBFFT_ERR_OOM;
    }
    if (p->rv->smem > 48 * 1024) {
        if (cudaFuncSetAttribute(p->rv->kfwd, cudaFuncAttributeMaxDynamicSharedMemorySize, p->rv->smem) !=
                cudaSuccess ||
            cudaFuncSetAttribute(p->rv->kinv, cudaFuncAttributeMaxDynamicSharedMemorySize, p->rv->smem) !=
                cudaSuccess) {
            free_plan(p);
            return GBFFT_ERR_CUDA;
        }
    }
    // Tables are built on the legacy stream and completed before the plan is returned.
    if (cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess ||
        launch_twiddle_table(p->tw, n, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        free_plan(p);
        return GBFFT_ERR_CUDA;
    }
    *out = p;
    return GBFFT_OK;
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
    return create(out, n, batch, direction, dtype, -1);
}

gbfft_status gbfft_plan_create_variant(gbfft_plan* out, int64_t n, int64_t batch, int direction, int dtype,
                                       int variant) {
    if (variant < 0) return GBFFT_ERR_NOT_FOUND;
    return create(out, n, batch, direction, dtype, variant);
}

gbfft_status gbfft_execute(gbfft_plan p, const void* in, void* out, void* cuda_stream) {
    if (!p) return GBFFT_ERR_INVALID_ARG;
    if (p->batch == 0) return GBFFT_OK;
    const size_t bytes = sizeof(float2) * (size_t)p->n * (size_t)p->batch;
    gbfft_status st = check_io(in, out, bytes);
    if (st != GBFFT_OK) return st;
    cudaError_t e = launch_rows(*p->rv, p->direction, (const float2*)in, (float2*)out, p->tw,
                                (long long)p->batch, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? GBFFT_OK : GBFFT_ERR_CUDA;
}

// Chunked host -> device -> host pipeline over a ring of staging buffers:
// while chunk c is transformed on the caller's stream, chunk c+1 is being
// copied in and chunk c-1 copied out on two internal streams.
gbfft_status gbfft_execute_host(gbfft_plan p, const void* host_in, void* host_out, void* cuda_stream) {
    if (!p || !host_in || !host_out) return GBFFT_ERR_INVALID_ARG;
    if (p->batch == 0) return GBFFT_OK;
    const size_t row_bytes = sizeof(float2) * (size_t)p->n;
    const size_t bytes = row_bytes * (size_t)p->batch;
    if (host_in != host_out) {
        const uintptr_t a = (uintptr_t)host_in, b = (uintptr_t)host_out;
        if (a < b + bytes && b < a + bytes) return GBFFT_ERR_OVERLAP;
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
    bool ok = cudaEventRecord(p->ev_start, su) == cudaSuccess && cudaStreamWaitEvent(p->s_in, p->ev_start, 0) == cudaSuccess;
    int used = 0;
    for (int64_t r0 = 0, c = 0; ok && r0 < p->batch; r0 += p->stage_rows, ++c) {
        const int b = (int)(c % gbfft_plan_s::kRing);
        const int64_t rows = (p->batch - r0) < p->stage_rows ? (p->batch - r0) : p->stage_rows;
        const size_t off = (size_t)r0 * row_bytes, nb = (size_t)rows * row_bytes;
        if (c >= gbfft_plan_s::kRing) ok = ok && cudaStreamWaitEvent(p->s_in, p->ev_out[b], 0) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(p->stage[b], hin + off, nb, cudaMemcpyHostToDevice, p->s_in) == cudaSuccess;
        ok = ok && cudaEventRecord(p->ev_in[b], p->s_in) == cudaSuccess;
        ok = ok && cudaStreamWaitEvent(su, p->ev_in[b], 0) == cudaSuccess;
        ok = ok && launch_rows(*p->rv, p->direction, p->stage[b], p->stage[b], p->tw, (long long)rows, su) ==
                       cudaSuccess;
        ok = ok && cudaEventRecord(p->ev_comp[b], su) == cudaSuccess;
        ok = ok && cudaStreamWaitEvent(p->s_out, p->ev_comp[b], 0) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(hout + off, p->stage[b], nb, cudaMemcpyDeviceToHost, p->s_out) == cudaSuccess;
        ok = ok && cudaEventRecord(p->ev_out[b], p->s_out) == cudaSuccess;
        if (used < gbfft_plan_s::kRing) ++used;
    }
    for (int b = 0; ok && b < used; ++b) ok = cudaStreamWaitEvent(su, p->ev_out[b], 0) == cudaSuccess;
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
    if (nstages) *nstages = p->rv->nstages;
    if (radices)
        for (int i = 0; i < p->rv->nstages; ++i) radices[i] = p->rv->radix[i];
    if (variant) *variant = p->variant;
    if (workspace_bytes) *workspace_bytes = p->ws_bytes;
    return GBFFT_OK;
}

int gbfft_num_variants(int64_t n) { return rows_variants_for(n, nullptr, 0); }

gbfft_status gbfft_variant_info(int64_t n, int index, int* nstages, int* radices, int* rows_per_cta,
                                int* threads_per_cta, int* smem_bytes) {
    const RowsVariant* cands[kMaxVariantsPerSize];
    const int nc = rows_variants_for(n, cands, kMaxVariantsPerSize);
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
