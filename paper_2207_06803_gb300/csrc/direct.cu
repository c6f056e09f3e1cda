// Direct DFT on the tensor cores for small N (the paper's "direct DFT"
// variant, which beat its recursive Cooley-Tukey for small sizes, Sec. VI):
// y = F_N x with F_N[m][q] = w_N^(m q), computed for 128 transforms at a time
// as one real matrix product
//     [yr yi] = [xr xi] [[Fr, Fi], [-Fi, Fr]]   (row vectors; K = 2N),
// i.e. D = A B^T with A = [xr xi] (128 x 2N, one transform per row) and B the
// 2N x 2N real form of F_N (row n_out: [Fr[n] | -Fi[n]] for the real parts,
// [Fi[n] | Fr[n]] for the imaginary parts).  Operands are split into high and
// low half-precision parts and D = Al Bh^T + Ah Bl^T + Ah Bh^T accumulates in
// FP32 in tensor memory (tcgen05.mma kind::f16, M = 128, N = K = 2N); FP16
// operands are first scaled by an exact power of two per transform.  No
// factorisation is needed, so every N that is a multiple of 8 up to 64 works.
//
// Per tile (128, 256 or 512 transforms: one to four M = 128 blocks, one thread
// per transform): threads load the rows with coalesced 16-byte loads (8 complex
// per chunk), split them into the K-major A operands in shared memory, one
// thread issues the MMAs and commits them to an mbarrier (bounded wait), each
// warp reads its 32 rows of D back from tensor memory, and the rows leave
// through a padded shared staging tile with coalesced 16-byte stores.  CTAs are
// persistent; B stays resident in shared memory, tensor memory is allocated
// once per CTA.  On a wait timeout the kernel records GBFFT_ERR_TIMEOUT, frees
// its tensor memory and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "tcgen05.cuh"

namespace gbfft {
namespace {

constexpr unsigned long long kDirectWaitNs = 1000000000ull;
constexpr int kDirectRows = 128;  // transforms per MMA block (the MMA's M)

constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }
constexpr uint32_t tmem_cols_for(int k) { return k <= 32 ? 32u : (k <= 64 ? 64u : (k <= 128 ? 128u : 256u)); }

template <int N>
struct DirectGeom {
    // 128-row blocks per tile (M = 128 MMAs): the choice that maximises resident warps per SM under the
    // shared-memory (A operands or output staging, plus B) and tensor-memory budgets
    static constexpr int BLK = N == 8 ? 4 : ((N == 16 || N == 40 || N == 64) ? 2 : 1);
    static constexpr int ROWS = kDirectRows * BLK;               // transforms per tile = threads per CTA
    static constexpr int K = 2 * N;                              // [re parts | im parts]
    static constexpr int LBO = 128;                              // K-adjacent core matrices
    static constexpr int SBO = 16 * K;                           // 8-row groups: K/8 core matrices of 128 B
    static constexpr int A_BYTES = kDirectRows * K * 2;          // one block's operand (hi or lo), halves
    static constexpr int B_BYTES = 2 * K * K * 2;                // [Bh; Bl]: 2K rows of K halves
    static constexpr int PITCH = 8 * N + 16;                     // staging row pitch (bytes), conflict-free
    static constexpr int AREG = round_up(cmax(2 * BLK * A_BYTES, ROWS * PITCH), 1024);
    static constexpr int SMEM = AREG + B_BYTES + ROWS * 4 + 16;
    static constexpr uint32_t COLS = tmem_cols_for(BLK * K);
    static_assert(N % 8 == 0 && BLK * K <= 256, "direct DFT: N a multiple of 8, tile columns <= 256");
};

// 32 bytes (8 floats) from a 32-byte-aligned global address in one request.
__device__ __forceinline__ void ld_global_v8(const float4* p, float (&w)[8]) {
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(w[0]), "=f"(w[1]), "=f"(w[2]), "=f"(w[3]), "=f"(w[4]), "=f"(w[5]), "=f"(w[6]), "=f"(w[7])
                 : "l"(p));
}

__device__ __forceinline__ uint32_t k_offset(int row, int kg, int sbo) {
    return (uint32_t)((row >> 3) * sbo + kg * 128 + (row & 7) * 16);
}

// V8: the input is 32-byte aligned (every chunk then is) and is read with 32-byte loads.
template <int N, int S, int PREC, bool V8>
__global__ void __launch_bounds__(DirectGeom<N>::ROWS) k_dft_direct_umma(const float2* in, float2* out,
                                                                         const uint4* __restrict__ bmat,
                                                                         long long batch, int* status) {
    using Geo = DirectGeom<N>;
    constexpr int K = Geo::K, BLK = Geo::BLK, ROWS = Geo::ROWS, CPR = N / 8;  // 8-complex chunks per row
    constexpr int G = CPR <= 1 ? 1 : (CPR <= 2 ? 2 : (CPR <= 4 ? 4 : 8));  // chunk slots per row (power of 2)
    constexpr int LPR = G < 4 ? G : 4, H = G / LPR;                          // lanes per row, chunks per lane
    extern __shared__ __align__(1024) uint8_t dsm[];
    uint8_t* const a_hi = dsm;                         // BLK blocks of 128 x K halves
    uint8_t* const a_lo = dsm + BLK * Geo::A_BYTES;
    uint8_t* const stage = dsm;  // output staging reuses the A region once the MMAs are done
    uint8_t* const bsm = dsm + Geo::AREG;
    int* const s_exp = reinterpret_cast<int*>(bsm + Geo::B_BYTES);
    uint64_t* const bar = reinterpret_cast<uint64_t*>(s_exp + ROWS);
    uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x;

    for (int i = tid; i < Geo::B_BYTES / 16; i += ROWS) reinterpret_cast<uint4*>(bsm)[i] = bmat[i];
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(Geo::COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    uint32_t phase = 0;
    bool ok = true;
    const long long ntiles = (batch + ROWS - 1) / ROWS;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();  // the previous tile's staging reads are done
        const long long r0 = tile * ROWS;
        const int nvalid = (int)min((long long)ROWS, batch - r0);
        const float4* src = reinterpret_cast<const float4*>(in + r0 * N);
        // Load, scale and split.  A row's G chunks (8 complex each) are held by LPR
        // lanes of one warp (H chunks per lane); a quarter-warp (8 lanes) covers 8
        // consecutive rows with the same chunk index, so its 16-byte stores into the
        // core-matrix layout (16 bytes per row per core matrix) hit 8 distinct bank
        // groups, and the row's lanes are 8 apart for the shuffle reduction.
        {
            const int lane = tid & 31, warp = tid >> 5;
            const int b8 = lane & 7, q = lane >> 3;
#pragma unroll
            for (int it = 0; it < LPR; ++it) {
                const int row = it * (ROWS / LPR) + warp * (32 / LPR) + b8 + 8 * (q / LPR);
                float re[H][8], im[H][8];
                float m = 0.f;
#pragma unroll
                for (int hh = 0; hh < H; ++hh) {
                    const int j = q % LPR + LPR * hh;
                    if constexpr (V8) {
                        // 32-byte loads: each request covers whole sectors
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            float w[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                            if (j < CPR && row < nvalid) ld_global_v8(src + (row * N + 8 * j) / 2 + 2 * h, w);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                re[hh][4 * h + e] = w[2 * e];
                                im[hh][4 * h + e] = w[2 * e + 1];
                            }
                        }
                    } else {
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (j < CPR && row < nvalid) v = src[(row * N + 8 * j) / 2 + h];
                            re[hh][2 * h] = v.x;
                            im[hh][2 * h] = v.y;
                            re[hh][2 * h + 1] = v.z;
                            im[hh][2 * h + 1] = v.w;
                        }
                    }
#pragma unroll
                    for (int e = 0; e < 8; ++e) m = fmaxf(m, fmaxf(fabsf(re[hh][e]), fabsf(im[hh][e])));
                }
                float sc = 1.f;
                if constexpr (PREC == 0) {
                    // exact power-of-two scale per row to [2^14, 2^15) (FP16 range)
#pragma unroll
                    for (int off = 8; off < 8 * LPR; off <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
                    int ex = (int)((__float_as_uint(m) >> 23) & 0xff) - 127;
                    if (!(m > 0.f)) ex = 0;
                    ex = max(-100, min(100, ex));
                    if (q % LPR == 0) s_exp[row] = ex;
                    sc = __uint_as_float((uint32_t)(127 + 14 - ex) << 23);
                }
                const uint32_t blk = (uint32_t)(row / kDirectRows) * Geo::A_BYTES;
                const int rr = row % kDirectRows;
#pragma unroll
                for (int hh = 0; hh < H; ++hh) {
                    const int j = q % LPR + LPR * hh;
                    if (j < CPR) {
                        uint32_t hr[4], lr[4], hi_[4], li[4];
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            float a, b;
                            hr[p] = pack_hi<PREC>(re[hh][2 * p] * sc, re[hh][2 * p + 1] * sc, a, b);
                            lr[p] = pack_lo<PREC>(a, b);
                            hi_[p] = pack_hi<PREC>(im[hh][2 * p] * sc, im[hh][2 * p + 1] * sc, a, b);
                            li[p] = pack_lo<PREC>(a, b);
                        }
                        const uint32_t o_re = blk + k_offset(rr, j, Geo::SBO);
                        const uint32_t o_im = blk + k_offset(rr, N / 8 + j, Geo::SBO);
                        *reinterpret_cast<uint4*>(a_hi + o_re) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
                        *reinterpret_cast<uint4*>(a_lo + o_re) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
                        *reinterpret_cast<uint4*>(a_hi + o_im) = make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
                        *reinterpret_cast<uint4*>(a_lo + o_im) = make_uint4(li[0], li[1], li[2], li[3]);
                    }
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            const uint32_t idesc = tc_instr_desc(PREC, kDirectRows, K);
            const uint32_t bh = smem_u32(bsm), bl = bh + (uint32_t)(K / 8) * Geo::SBO;  // rows K..2K-1 = Bl
#pragma unroll
            for (int b = 0; b < BLK; ++b) {
                const uint32_t d = tmem + (uint32_t)(b * K);
                const uint32_t ah = smem_u32(a_hi + b * Geo::A_BYTES), al = smem_u32(a_lo + b * Geo::A_BYTES);
                // D = Al Bh^T + Ah Bl^T + Ah Bh^T (small terms first), K = 16 per instruction
#pragma unroll
                for (int ks = 0; ks < K / 16; ++ks)
                    tc_mma_f16(d, tc_smem_desc(al + ks * 256, Geo::LBO, Geo::SBO),
                               tc_smem_desc(bh + ks * 256, Geo::LBO, Geo::SBO), idesc, ks);
#pragma unroll
                for (int ks = 0; ks < K / 16; ++ks)
                    tc_mma_f16(d, tc_smem_desc(ah + ks * 256, Geo::LBO, Geo::SBO),
                               tc_smem_desc(bl + ks * 256, Geo::LBO, Geo::SBO), idesc, 1);
#pragma unroll
                for (int ks = 0; ks < K / 16; ++ks)
                    tc_mma_f16(d, tc_smem_desc(ah + ks * 256, Geo::LBO, Geo::SBO),
                               tc_smem_desc(bh + ks * 256, Geo::LBO, Geo::SBO), idesc, 1);
            }
            tc_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait(bar, phase, kDirectWaitNs) ? 1 : 0);
        phase ^= 1u;
        if (!ok) break;
        tc_fence_after();
        // Row tid of the tile: warp w reads TMEM lanes 32 (w % 4) .. + 31 of block w / 4.
        const int row = tid, warp = tid >> 5;
        const float inv_sc = PREC == 0 ? __uint_as_float((uint32_t)(127 - 14 + s_exp[row]) << 23) : 1.f;
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * K);
        float4* srow = reinterpret_cast<float4*>(stage + row * Geo::PITCH);
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 8) {
            float yr[8], yi[8];
            tmem_ld8(taddr + (uint32_t)c0, yr);
            tmem_ld8(taddr + (uint32_t)(N + c0), yi);
#pragma unroll
            for (int h = 0; h < 4; ++h)
                srow[c0 / 2 + h] = make_float4(yr[2 * h] * inv_sc, yi[2 * h] * inv_sc, yr[2 * h + 1] * inv_sc,
                                               yi[2 * h + 1] * inv_sc);
        }
        tc_fence_before();
        __syncthreads();
        float4* dst = reinterpret_cast<float4*>(out + r0 * N);
        constexpr int PPR = N / 2;  // 16-byte pieces per row
#pragma unroll
        for (int i = 0; i < PPR; ++i) {
            const int p = tid + i * ROWS;
            const int r = p / PPR;
            if (r < nvalid) dst[p] = *reinterpret_cast<const float4*>(stage + r * Geo::PITCH + (p % PPR) * 16);
        }
    }
    if (!ok && tid == 0) atomicCAS(status, 0, (int)GBFFT_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Geo::COLS) : "memory");
}

// B = [Bh; Bl] (2K rows of K halves, K-major core-matrix layout): row n < K is
// the high part of [Fr[n] | -Fi[n]] (n < N) or [Fi[n-N] | Fr[n-N]] (n >= N),
// row K + n its low part; F[m][q] = exp(sign 2 pi i m q / N) in FP64.
__global__ void k_direct_bmat(uint16_t* bm, int n, int prec, int sign) {
    const int k2 = 2 * n, sbo = 16 * k2;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // row * K + kk
    if (idx >= 2 * k2 * k2) return;
    const int row = idx / k2, kk = idx % k2;
    const int part = row / k2, nr = row % k2;
    const int m = nr % n, q = kk % n;
    const int e = (m * q) % n;
    double sn, cs;
    sincospi(2.0 * (double)e / (double)n, &sn, &cs);
    const double fr = cs, fi = (double)sign * sn;
    double v;
    if (nr < n) v = kk < n ? fr : -fi;
    else v = kk < n ? fi : fr;
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
    const uint32_t off = (uint32_t)((row >> 3) * sbo + (kk >> 3) * 128 + (row & 7) * 16 + (kk & 7) * 2);
    bm[off / 2] = bits;
}

template <int N>
DirectVariant make_direct_variant() {
    DirectVariant v{};
    v.n = N;
    v.rows = DirectGeom<N>::ROWS;
    v.tpb = DirectGeom<N>::ROWS;
    v.smem = DirectGeom<N>::SMEM;
    v.bmat_bytes = DirectGeom<N>::B_BYTES;
    v.tmem_cols = (int)DirectGeom<N>::COLS;
    v.k[0][0] = (const void*)&k_dft_direct_umma<N, -1, 0, false>;
    v.k[0][1] = (const void*)&k_dft_direct_umma<N, +1, 0, false>;
    v.k[1][0] = (const void*)&k_dft_direct_umma<N, -1, 1, false>;
    v.k[1][1] = (const void*)&k_dft_direct_umma<N, +1, 1, false>;
    v.k32[0][0] = (const void*)&k_dft_direct_umma<N, -1, 0, true>;
    v.k32[0][1] = (const void*)&k_dft_direct_umma<N, +1, 0, true>;
    v.k32[1][0] = (const void*)&k_dft_direct_umma<N, -1, 1, true>;
    v.k32[1][1] = (const void*)&k_dft_direct_umma<N, +1, 1, true>;
    return v;
}

const DirectVariant kDirect[] = {
    make_direct_variant<8>(),  make_direct_variant<16>(), make_direct_variant<24>(), make_direct_variant<32>(),
    make_direct_variant<40>(), make_direct_variant<48>(), make_direct_variant<56>(), make_direct_variant<64>(),
};

}  // namespace

const DirectVariant* direct_variant_for(int64_t n) {
    for (const DirectVariant& v : kDirect)
        if (v.n == n) return &v;
    return nullptr;
}

cudaError_t prepare_direct(const DirectVariant& v) {
    for (int p = 0; p < 2; ++p)
        for (int d = 0; d < 2; ++d) {
            cudaError_t e = cudaFuncSetAttribute(v.k[p][d], cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(v.k32[p][d], cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

// Resident CTAs per SM from the kernel's registers, shared memory, threads and
// tensor-memory columns (512 per SM), times the SM count.
int direct_grid(const DirectVariant& v) {
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
    per_sm = std::min(per_sm, 512 / v.tmem_cols);
    per_sm = std::min(per_sm, prop.maxBlocksPerMultiProcessor);
    return per_sm < 1 ? 0 : per_sm * prop.multiProcessorCount;
}

cudaError_t launch_direct_bmat(uint16_t* bm, int n, int prec, int sign, cudaStream_t s) {
    const int total = 2 * (2 * n) * (2 * n);
    k_direct_bmat<<<(total + 255) / 256, 256, 0, s>>>(bm, n, prec, sign);
    return cudaGetLastError();
}

cudaError_t launch_direct(const DirectVariant& v, int prec, int direction, const float2* in, float2* out,
                          const void* bmat, long long batch, int grid_cap, int* status, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    long long blocks = (batch + v.rows - 1) / v.rows;
    if (grid_cap > 0 && blocks > grid_cap) blocks = grid_cap;
    void* args[] = {(void*)&in, (void*)&out, (void*)&bmat, (void*)&batch, (void*)&status};
    const bool a32 = ((uintptr_t)in & 31u) == 0;  // 32-byte loads need a 32-byte-aligned input
    const void* fn = (a32 ? v.k32 : v.k)[prec][direction == GBFFT_FORWARD ? 0 : 1];
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(v.tpb), args, (size_t)v.smem, s);
}

}  // namespace gbfft
