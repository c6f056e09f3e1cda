// Tensor-core variant on the fifth-generation tensor cores (tcgen05, TMEM).
//
// Same arithmetic as tc.cu (every radix-16 stage's DFT_16 as the real product
// [yr; yi] = M [xr; xi], M = [[Fr, -Fi], [Fi, Fr]], with operands split into
// high and low half-precision parts, Mh Xh + Mh Xl + Ml Xh, FP32 accumulation),
// arranged for tcgen05.mma instead of warp-level mma.sync:
//   - each CTA's next tile of rows is copied HBM -> shared memory by a bulk
//     copy (cp.async.bulk, completing on an mbarrier) issued as soon as the
//     first stage has read the current tile, so the load overlaps the
//     remaining stages;
//   - one thread per butterfly (column of 16 complex), exactly as the FP32
//     Stockham engine: it loads its column, applies the FP32 stage twiddles,
//     scales by an exact power of two (FP16), splits into hi/lo and writes
//     the column as one 32-element row of the A operands Ah = Xh^T and
//     Al = Xl^T (128 rows per MMA tile) in shared memory;
//   - B = [Mh; Ml]^T is resident in shared memory for the whole kernel;
//   - one elected thread issues D = Al Mh^T + Ah Ml^T + Ah Mh^T into the same
//     32 TMEM columns (N = 32, each product as two K = 16 instructions) and
//     commits them to an mbarrier; D (128 lanes x 32 FP32 columns per M tile)
//     lives in tensor memory;
//   - each warp reads back its own 32 TMEM lanes (its own 32 butterflies) with
//     tcgen05.ld, then writes the 16 outputs with the Stockham pattern
//     (shared-memory exchange or HBM).
// The A operands share their shared memory with the exchange buffer of the
// stages: a stage reads its columns from the exchange buffer, all threads
// meet at a barrier, and only then are the operands written over it; the
// outputs go back into it once the MMA has completed.
// Operand layout: K-major, no swizzle; a core matrix is 8 rows x 16 bytes
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
constexpr int kRowBytes = 64;    // one 32-element K row of halves
constexpr int kLbo = 128;        // K-adjacent core matrices
constexpr int kSbo = 512;        // 8-row groups (4 core matrices of K)
constexpr int kTileBytes = 128 * kRowBytes;  // one 128 x 32 operand

__device__ __forceinline__ uint32_t a_offset(int row, int kgroup) {
    return (uint32_t)((row >> 3) * kSbo + kgroup * kLbo + (row & 7) * 16);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) { return tc_smem_desc(saddr, kLbo, kSbo); }

__host__ __device__ constexpr uint32_t instr_desc(int prec, int m, int n) { return tc_instr_desc(prec, m, n); }

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    tc_mma_f16(tmem_d, adesc, bdesc, idesc, accumulate);
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) { tc_commit(bar); }

struct UmmaShared {
    float2* stage;       // the tile's input rows, natural order (bulk copy target)
    uint8_t* a_hi;       // MT tiles of 128 x 32, over the exchange buffer
    uint8_t* a_lo;
    uint8_t* b;          // [Mh; Ml] as 64 rows x 32 (K-major)
    float2* xbuf;        // padded exchange buffer
    uint64_t* bar;       // MMA completion
    uint64_t* ldbar;     // bulk copy of the next tile
    uint32_t* tmem_slot; // TMEM base address written by tcgen05.alloc
};

// The next tile's bulk copy, issued by thread 0 once the first stage has read the
// staging buffer (src == nullptr: no next tile).
struct NextTile {
    const float2* src;
    uint32_t bytes;
};

// One radix-16 stage: threads own butterflies B = tid (MT*128 of them).
template <int N, int S, int PREC, int T, int PS, int L, bool FIRST, bool LAST>
__device__ __forceinline__ bool umma_stage(const ContigIO<N>& io, const UmmaShared& sh, uint32_t tmem,
                                           const float2* __restrict__ tw, int nvalid, uint32_t& phase,
                                           const NextTile& next) {
    constexpr int R = 16, NR = N / R;
    const int tid = threadIdx.x;
    const int B = tid;
    const int t = B / NR, j = B % NR, k = j % L;
    float2 x[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int n = j + q * NR;
        if constexpr (FIRST) {
            x[q] = (t < nvalid) ? sh.stage[t * N + n] : make_float2(0.f, 0.f);
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
    // The operands overwrite the exchange buffer: every thread has read its column first.
    if constexpr (!FIRST) __syncthreads();
    // Row B of Ah / Al: K index 0..15 = real parts (q), 16..31 = imaginary parts.
    {
        const int mt = B >> 7, row = B & 127;
        uint8_t* ah = sh.a_hi + mt * kTileBytes;
        uint8_t* al = sh.a_lo + mt * kTileBytes;
#pragma unroll
        for (int kg = 0; kg < 4; ++kg) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int kk = kg * 8 + 2 * p;  // K index of the pair's first element
                const float a0 = kk < 16 ? x[kk].x : x[kk - 16].y;
                const float a1 = kk < 16 ? x[kk + 1].x : x[kk - 15].y;
                float r0, r1;
                h[p] = pack_hi<PREC>(a0, a1, r0, r1);
                l[p] = pack_lo<PREC>(r0, r1);
            }
            *reinterpret_cast<uint4*>(ah + a_offset(row, kg)) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(al + a_offset(row, kg)) = make_uint4(l[0], l[1], l[2], l[3]);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    constexpr int MT = T * N / 16 / 128;
    if (tid == 0) {
        if constexpr (FIRST) {
            // every thread has read the staging buffer: bring in the next tile behind the stages
            if (next.src) {
                fence_proxy_async_smem();
                mbar_expect_tx(sh.ldbar, next.bytes);
                tma_load_1d(sh.stage, next.src, next.bytes, sh.ldbar);
            }
        }
        const uint32_t idesc = instr_desc(PREC, 128, 32);
        const uint32_t b_mh = smem_u32(sh.b), b_ml = b_mh + 4 * kSbo;  // rows 0-31 = Mh, 32-63 = Ml
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const uint32_t d = tmem + (uint32_t)(mt * 32);
            const uint32_t ah = smem_u32(sh.a_hi + mt * kTileBytes), al = smem_u32(sh.a_lo + mt * kTileBytes);
            // D = Al Mh^T + Ah Ml^T + Ah Mh^T (small terms first), each as two K = 16 steps
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                umma_f16(d, smem_desc(al + ks * 2 * kLbo), smem_desc(b_mh + ks * 2 * kLbo), idesc, ks);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                umma_f16(d, smem_desc(ah + ks * 2 * kLbo), smem_desc(b_ml + ks * 2 * kLbo), idesc, 1);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                umma_f16(d, smem_desc(ah + ks * 2 * kLbo), smem_desc(b_mh + ks * 2 * kLbo), idesc, 1);
        }
        umma_commit(sh.bar);
    }
    const int ok = __syncthreads_and(mbar_wait(sh.bar, phase, kUmmaWaitNs) ? 1 : 0);
    phase ^= 1u;
    if (!ok) return false;
    tc_fence_after();
    // Warp w reads TMEM lanes 32*(w%4) .. +31 of the D tile of its M-tile.
    const int warp = tid >> 5;
    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 32);
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
                                            const float2* __restrict__ tw, int nvalid, uint32_t& phase,
                                            const NextTile& next) {
    constexpr bool LAST = (L * 16 == N);
    if (!umma_stage<N, S, PREC, T, PS, L, L == 1, LAST>(io, sh, tmem, tw + (L > 1 ? L - 16 : 0), nvalid, phase,
                                                        next))
        return false;
    if constexpr (!LAST) return umma_stages<N, S, PREC, T, PS, L * 16>(io, sh, tmem, tw, nvalid, phase, next);
    return true;
}

template <int N, int T, int PS>
constexpr int umma_union_bytes() {
    constexpr int a = 2 * (T * N / 16 / 128) * kTileBytes;
    constexpr int x = smem_elems<T, N, PS>() * 8;
    return ((a > x ? a : x) + 1023) / 1024 * 1024;
}

// bmat: 64 x 32 halves in the K-major core-matrix layout (k_umma_bmat).
template <int N, int S, int PREC, int T, int PS>
__global__ void __launch_bounds__(T * N / 16) k_stockham_umma(const float2* in, float2* out,
                                                               const float2* __restrict__ tw,
                                                               const uint4* __restrict__ bmat, long long batch,
                                                               int* status) {
    constexpr int TPB = T * N / 16;
    constexpr int MT = TPB / 128;
    constexpr uint32_t kCols = MT == 1 ? 32 : 64;
    static_assert(TPB % 128 == 0 && (MT == 1 || MT == 2), "one or two M = 128 tiles per stage");
    constexpr int kStageBytes = T * N * 8;
    constexpr int kUnionBytes = umma_union_bytes<N, T, PS>();
    extern __shared__ __align__(1024) uint8_t usm[];
    UmmaShared sh;
    sh.stage = reinterpret_cast<float2*>(usm);
    sh.a_hi = usm + kStageBytes;
    sh.a_lo = sh.a_hi + MT * kTileBytes;
    sh.xbuf = reinterpret_cast<float2*>(sh.a_hi);
    sh.b = usm + kStageBytes + kUnionBytes;
    sh.bar = reinterpret_cast<uint64_t*>(sh.b + 64 * kRowBytes);
    sh.ldbar = sh.bar + 1;
    sh.tmem_slot = reinterpret_cast<uint32_t*>(sh.bar + 2);
    const int tid = threadIdx.x;
    // B operand, resident for the kernel (64 rows x 64 bytes = 256 uint4).
    for (int i = tid; i < 64 * kRowBytes / 16; i += TPB) reinterpret_cast<uint4*>(sh.b)[i] = bmat[i];
    if (tid == 0) {
        mbar_init(sh.bar, 1);
        mbar_init(sh.ldbar, 1);
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
    uint32_t phase = 0, ldphase = 0;
    const long long ntiles = (batch + T - 1) / T;
    if (tid == 0 && blockIdx.x < ntiles) {
        const uint32_t bytes = (uint32_t)(tile_rows(blockIdx.x, T, batch) * N * 8);
        mbar_expect_tx(sh.ldbar, bytes);
        tma_load_1d(sh.stage, in + (long long)blockIdx.x * T * N, bytes, sh.ldbar);
    }
    bool ok = true;
    for (long long tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        ok = __syncthreads_and(mbar_wait(sh.ldbar, ldphase, kUmmaWaitNs) ? 1 : 0);
        if (!ok) break;  // the only copy in flight is the one that did not arrive
        ldphase ^= 1u;
        const int nvalid = tile_rows(tile, T, batch);
        const long long nt = tile + gridDim.x;
        const NextTile next{nt < ntiles ? in + nt * T * N : nullptr,
                            nt < ntiles ? (uint32_t)(tile_rows(nt, T, batch) * N * 8) : 0u};
        const ContigIO<N> io{nullptr, out + tile * T * N};
        ok = umma_stages<N, S, PREC, T, PS, 1>(io, sh, tmem, tw, nvalid, phase, next);
        // the first stage issued the next tile's copy before any wait that can fail: let it land
        if (!ok && next.src) mbar_wait(sh.ldbar, ldphase, kUmmaWaitNs);
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
    return T * N * 8 + umma_union_bytes<N, T, PS>() + 64 * kRowBytes + 32;
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
    per_sm = std::min(per_sm, 512 / (v.tpb > 128 ? 64 : 32));  // TMEM columns
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
