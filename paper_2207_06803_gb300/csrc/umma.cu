// Tensor-core variant on the fifth-generation tensor cores (tcgen05, TMEM).
//
// Same arithmetic as tc.cu (every radix-16 stage's DFT_16 as the real product
// [yr; yi] = M [xr; xi], M = [[Fr, -Fi], [Fi, Fr]], with operands split into
// high and low half-precision parts, Mh Xh + Mh Xl + Ml Xh, FP32 accumulation),
// arranged for tcgen05.mma instead of warp-level mma.sync:
//   - one thread per butterfly (column of 16 complex), exactly as the FP32
//     Stockham engine: it loads its column (HBM in the first stage, the
//     exchange buffer after), applies the FP32 stage twiddles, scales by an
//     exact power of two (FP16), splits into hi/lo and stores the column as
//     row B of the A operands Ah = Xh^T and Al = Xl^T straight into TENSOR
//     memory (tcgen05.st: each thread writes its own lane, 16 columns of
//     packed halves per part) - the operands never touch shared memory, so a
//     stage moves 16 bytes per point through shared memory, as the FP32 engine
//     does (operands in shared memory took 36 and bounded the kernel there);
//   - B = [Mh; Ml]^T is resident in shared memory for the whole kernel;
//   - one elected thread issues D = Al Mh^T + Ah Ml^T + Ah Mh^T with A read
//     from tensor memory (N = 32, each product as two K = 16 instructions) and
//     commits them to an mbarrier; per M = 128 tile, tensor memory holds D in
//     columns 0..31, Ah in 32..47 and Al in 48..63;
//   - each warp reads back its own 32 TMEM lanes (its own 32 butterflies) with
//     tcgen05.ld, then writes the 16 outputs with the Stockham pattern
//     (shared-memory exchange or HBM).
// B operand layout: K-major, no swizzle; a core matrix is 8 rows x 16 bytes
// (8 halves of K), core matrices adjacent in K are 128 bytes apart (leading
// byte offset) and 8-row groups 512 bytes apart (stride byte offset).
// Every wait is bounded (globaltimer deadline); on expiry the kernel records
// GBFFT_ERR_TIMEOUT, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "stockham.cuh"
#include "tcgen05.cuh"

namespace gbfft {
namespace {

constexpr unsigned long long kUmmaWaitNs = 1000000000ull;
constexpr int kRowBytes = 64;    // one 32-element K row of halves (B operand)
constexpr int kLbo = 128;        // K-adjacent core matrices
constexpr int kSbo = 512;        // 8-row groups (4 core matrices of K)

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) { return tc_smem_desc(saddr, kLbo, kSbo); }

__host__ __device__ constexpr uint32_t instr_desc(int prec, int m, int n) { return tc_instr_desc(prec, m, n); }

__device__ __forceinline__ void umma_commit(uint64_t* bar) { tc_commit(bar); }

struct UmmaShared {
    uint8_t* b;          // [Mh; Ml] as 64 rows x 32 (K-major)
    float2* xbuf;        // padded exchange buffer
    uint64_t* bar;       // MMA completion
    uint32_t* tmem_slot; // TMEM base address written by tcgen05.alloc
};

// One radix-16 stage: threads own butterflies B = tid (MT*128 of them).
template <int N, int S, int PREC, int T, int PS, int L, bool FIRST, bool LAST>
__device__ __forceinline__ bool umma_stage(const ContigIO<N>& io, const UmmaShared& sh, uint32_t tmem,
                                           const float2* __restrict__ tw, int nvalid, uint32_t& phase) {
    constexpr int R = 16, NR = N / R;
    const int tid = threadIdx.x;
    const int B = tid;
    const int t = B / NR, j = B % NR, k = j % L;
    float2 x[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int n = j + q * NR;
        if constexpr (FIRST) {
            x[q] = (t < nvalid) ? io.ld(t, n) : make_float2(0.f, 0.f);
        } else {
            x[q] = sh.xbuf[spad<PS>(t * N + n)];
        }
    }
    if constexpr (L > 1) {
        float2 w[16];
        twiddle_powers16(tw, L, k, w);  // four table reads, the other powers by products
#pragma unroll
        for (int q = 1; q < 16; ++q) x[q] = twiddle<S>(x[q], w[q]);
    }
    float inv_sc = 1.f;
    if constexpr (PREC == 0) {
        float m = 0.f;
#pragma unroll
        for (int q = 0; q < 16; ++q) m = fmaxf(m, fmaxf(fabsf(x[q].x), fabsf(x[q].y)));
        int e = (int)((__float_as_uint(m) >> 23) & 0xff) - 127;
        if (!(m > 0.f)) e = 0;
        e = max(-100, min(100, e));
        const float sc = __uint_as_float((uint32_t)(127 + 14 - e) << 23);
        inv_sc = __uint_as_float((uint32_t)(127 - 14 + e) << 23);
#pragma unroll
        for (int q = 0; q < 16; ++q) x[q] = make_float2(x[q].x * sc, x[q].y * sc);
    }
    // Row B of Ah / Al into tensor memory (lane = row of this warp's sub-partition): K index 0..15 = real
    // parts (q), 16..31 = imaginary parts, two halves per column; M tile mt holds D at columns mt*64 + 0..31,
    // Ah at + 32..47, Al at + 48..63.
    constexpr int MT = T * N / 16 / 128;
    const int warp = tid >> 5, mt = warp >> 2;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
#pragma unroll
    for (int part = 0; part < 2; ++part) {  // real parts (K 0..15), then imaginary parts (K 16..31)
        uint32_t h[8], l[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float a0 = part == 0 ? x[2 * c].x : x[2 * c].y;
            const float a1 = part == 0 ? x[2 * c + 1].x : x[2 * c + 1].y;
            float r0, r1;
            h[c] = pack_hi<PREC>(a0, a1, r0, r1);
            l[c] = pack_lo<PREC>(r0, r1);
        }
        tmem_st8(tmem + lane_base + (uint32_t)(mt * 64 + 32 + part * 8), h);
        tmem_st8(tmem + lane_base + (uint32_t)(mt * 64 + 48 + part * 8), l);
    }
    tmem_st_wait();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        const uint32_t idesc = instr_desc(PREC, 128, 32);
        const uint32_t b_mh = smem_u32(sh.b), b_ml = b_mh + 4 * kSbo;  // rows 0-31 = Mh, 32-63 = Ml
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            const uint32_t d = tmem + (uint32_t)(m * 64), ah = d + 32, al = d + 48;
            // D = Al Mh^T + Ah Ml^T + Ah Mh^T (small terms first), each as two K = 16 steps (8 columns of A)
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                tc_mma_f16_ta(d, al + (uint32_t)(ks * 8), smem_desc(b_mh + ks * 2 * kLbo), idesc, ks);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                tc_mma_f16_ta(d, ah + (uint32_t)(ks * 8), smem_desc(b_ml + ks * 2 * kLbo), idesc, 1);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                tc_mma_f16_ta(d, ah + (uint32_t)(ks * 8), smem_desc(b_mh + ks * 2 * kLbo), idesc, 1);
        }
        umma_commit(sh.bar);
    }
    const int ok = __syncthreads_and(mbar_wait(sh.bar, phase, kUmmaWaitNs) ? 1 : 0);
    phase ^= 1u;
    if (!ok) return false;
    tc_fence_after();
    // Warp w reads TMEM lanes 32*(w%4) .. +31 of the D tile of its M-tile.
    const uint32_t taddr = tmem + lane_base + (uint32_t)(mt * 64);
    float d0[32];
    tmem_ld32(taddr, d0);
    float2 y[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) y[m] = make_float2(d0[m] * inv_sc, d0[16 + m] * inv_sc);
    tc_fence_before();
    // the MMA has completed (every thread passed the wait), so the operands are dead and the
    // exchange buffer may take the outputs
    const int b = j / L;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        if constexpr (LAST) {
            if (t < nvalid) io.st(t, m * L + j, y[m]);
        } else {
            sh.xbuf[spad<PS>(t * N + b * L * R + m * L + k)] = y[m];
        }
    }
    if constexpr (!LAST) __syncthreads();
    return true;
}

template <int N, int S, int PREC, int T, int PS, int L>
__device__ __forceinline__ bool umma_stages(const ContigIO<N>& io, const UmmaShared& sh, uint32_t tmem,
                                            const float2* __restrict__ tw, int nvalid, uint32_t& phase) {
    constexpr bool LAST = (L * 16 == N);
    if (!umma_stage<N, S, PREC, T, PS, L, L == 1, LAST>(io, sh, tmem, tw + (L > 1 ? L - 16 : 0), nvalid, phase))
        return false;
    if constexpr (!LAST) return umma_stages<N, S, PREC, T, PS, L * 16>(io, sh, tmem, tw, nvalid, phase);
    return true;
}

template <int N, int T, int PS>
constexpr int umma_xbuf_bytes() {
    constexpr int x = smem_elems<T, N, PS>() * 8;
    return (x + 1023) / 1024 * 1024;
}

// bmat: 64 x 32 halves in the K-major core-matrix layout (k_umma_bmat).  Persistent
// CTAs walk tiles of T rows; 64 registers per thread (4 CTAs of 256 threads or 8 of
// 128 per SM, the tensor memory of four 128-column or eight 64-column allocations).
template <int N, int S, int PREC, int T, int PS>
__global__ void __launch_bounds__(T * N / 16, (T * N / 16) == 256 ? 4 : 8)
    k_stockham_umma(const float2* in, float2* out, const float2* __restrict__ tw, const uint4* __restrict__ bmat,
                    long long batch, int* status) {
    constexpr int TPB = T * N / 16;
    constexpr int MT = TPB / 128;
    constexpr uint32_t kCols = MT == 1 ? 64 : 128;  // per M tile: D 32 columns, Ah 16, Al 16
    static_assert(TPB % 128 == 0 && (MT == 1 || MT == 2), "one or two M = 128 tiles per stage");
    constexpr int kXbufBytes = umma_xbuf_bytes<N, T, PS>();
    extern __shared__ __align__(1024) uint8_t usm[];
    UmmaShared sh;
    sh.xbuf = reinterpret_cast<float2*>(usm);
    sh.b = usm + kXbufBytes;
    sh.bar = reinterpret_cast<uint64_t*>(sh.b + 64 * kRowBytes);
    sh.tmem_slot = reinterpret_cast<uint32_t*>(sh.bar + 1);
    const int tid = threadIdx.x;
    // B operand, resident for the kernel (64 rows x 64 bytes = 256 uint4).
    for (int i = tid; i < 64 * kRowBytes / 16; i += TPB) reinterpret_cast<uint4*>(sh.b)[i] = bmat[i];
    if (tid == 0) {
        mbar_init(sh.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sh.tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sh.tmem_slot;
    uint32_t phase = 0;
    const long long ntiles = (batch + T - 1) / T;
    bool ok = true;
    for (long long tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        __syncthreads();  // the previous tile's last readers of the exchange buffer are done
        const int nvalid = tile_rows(tile, T, batch);
        const ContigIO<N> io{in + tile * T * N, out + tile * T * N};
        ok = umma_stages<N, S, PREC, T, PS, 1>(io, sh, tmem, tw, nvalid, phase);
    }
    if (!ok && tid == 0) atomicCAS(status, 0, (int)GBFFT_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// B = [Mh; Ml]: row n < 32 is Mh row n, row 32 + n is Ml row n, K-major
// core-matrix layout; M[n][k] = [[Fr, -Fi], [Fi, Fr]][n][k] of
// F = exp(sign * 2 pi i n q / 16), evaluated in FP64 and split hi/lo.
__global__ void k_umma_bmat(uint16_t* bm, int prec, int sign) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // row * 32 + k
    if (idx >= 64 * 32) return;
    const int row = idx / 32, kk = idx % 32;
    const int part = row / 32, n = row % 32;
    const int m = n % 16, q = kk % 16;
    const int e = (m * q) % 16;
    double sn, cs;
    sincospi(2.0 * (double)e / 16.0, &sn, &cs);
    const double fr = cs, fi = (double)sign * sn;
    double v;
    if (n < 16) v = kk < 16 ? fr : -fi;
    else v = kk < 16 ? fi : fr;
    uint16_t bits;
    if (prec == 0) {
        const __half hi = __double2half(v);
        const __half lo = __double2half(v - (double)__half2float(hi));
        const __half pick = part == 0 ? hi : lo;
        bits = *reinterpret_cast<const uint16_t*>(&pick);
    } else {
        const __nv_bfloat16 hi = __double2bfloat16(v);
        const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
        const __nv_bfloat16 pick = part == 0 ? hi : lo;
        bits = *reinterpret_cast<const uint16_t*>(&pick);
    }
    const uint32_t off = (uint32_t)((row >> 3) * kSbo + (kk >> 3) * kLbo + (row & 7) * 16 + (kk & 7) * 2);
    bm[off / 2] = bits;
}

template <int N, int T, int PS>
constexpr int umma_smem_bytes() {
    return umma_xbuf_bytes<N, T, PS>() + 64 * kRowBytes + 32;
}

template <int N, int T, int PS>
UmmaVariant make_umma_variant() {
    UmmaVariant v{};
    v.n = N;
    v.rows = T;
    v.tpb = T * N / 16;
    v.smem = umma_smem_bytes<N, T, PS>();
    v.k[0][0] = (const void*)&k_stockham_umma<N, -1, 0, T, PS>;
    v.k[0][1] = (const void*)&k_stockham_umma<N, +1, 0, T, PS>;
    v.k[1][0] = (const void*)&k_stockham_umma<N, -1, 1, T, PS>;
    v.k[1][1] = (const void*)&k_stockham_umma<N, +1, 1, T, PS>;
    return v;
}

const UmmaVariant kUmma[] = {
    make_umma_variant<256, 8, 4>(),
    make_umma_variant<4096, 1, 4>(),
};

}  // namespace

const UmmaVariant* umma_variant_for(int64_t n) {
    for (const UmmaVariant& v : kUmma)
        if (v.n == n) return &v;
    return nullptr;
}

cudaError_t prepare_umma(const UmmaVariant& v) {
    for (int p = 0; p < 2; ++p)
        for (int d = 0; d < 2; ++d) {
            cudaError_t e = cudaFuncSetAttribute(v.k[p][d], cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

// Resident CTAs per SM from the kernel's own resources (registers, shared
// memory, threads) and its tensor-memory columns, times the SM count.
int umma_grid(const UmmaVariant& v) {
    int dev = 0;
    cudaDeviceProp prop;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, v.k[0][0]) != cudaSuccess)
        return 0;
    int per_sm = prop.maxThreadsPerMultiProcessor / v.tpb;
    const int regs = fa.numRegs > 0 ? fa.numRegs : 255;
    per_sm = std::min(per_sm, prop.regsPerMultiprocessor / (regs * v.tpb));
    const int smem = v.smem + (int)fa.sharedSizeBytes + 1024;  // + per-CTA reservation
    per_sm = std::min(per_sm, (int)prop.sharedMemPerMultiprocessor / smem);
    per_sm = std::min(per_sm, 512 / (v.tpb > 128 ? 128 : 64));  // TMEM columns
    per_sm = std::min(per_sm, prop.maxBlocksPerMultiProcessor);
    return per_sm < 1 ? 0 : per_sm * prop.multiProcessorCount;
}

cudaError_t launch_umma_bmat(uint16_t* bm, int prec, int sign, cudaStream_t s) {
    k_umma_bmat<<<8, 256, 0, s>>>(bm, prec, sign);
    return cudaGetLastError();
}

cudaError_t launch_umma(const UmmaVariant& v, int prec, int direction, const float2* in, float2* out,
                        const float2* tw, const void* bmat, long long batch, int grid_cap, int* status,
                        cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    long long blocks = (batch + v.rows - 1) / v.rows;
    if (grid_cap > 0 && blocks > grid_cap) blocks = grid_cap;
    void* args[] = {(void*)&in, (void*)&out, (void*)&tw, (void*)&bmat, (void*)&batch, (void*)&status};
    const void* fn = v.k[prec][direction == GBFFT_FORWARD ? 0 : 1];
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(v.tpb), args, (size_t)v.smem, s);
}

}  // namespace gbfft
