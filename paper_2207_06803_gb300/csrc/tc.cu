// Tensor-core variant: every radix-16 stage's DFT_16 runs as split-precision
// products on the tensor cores.
//
// A radix-16 stage applies DFT_16 to the (twiddled) 16-point columns of the
// stage.  Written over the reals, with a column x = xr + i xi and
// F = DFT_16 = Fr + i Fi,
//     [yr; yi] = [[Fr, -Fi], [Fi, Fr]] [xr; xi]      (a 32 x 32 real matrix M),
// so 8 columns at a time form one 32x32 . 32x8 product: two 16-row tiles
// (real and imaginary outputs) by two 16-deep tiles (real and imaginary
// inputs) of mma.m16n8k16 with FP32 accumulation.  Operands are split into a
// high and a low half-precision part, M = Mh + Ml and X = Xh + Xl, and the
// product is taken as Mh Xh + Mh Xl + Ml Xh (the Ml Xl term is dropped), which
// keeps about twice the half type's significand:
//   FP16: each column is first scaled by a power of two so that its largest
//         magnitude lies in [2^14, 2^15) (no overflow, no subnormal low parts);
//         the scale is exact and undone on the FP32 result.
//   BF16: FP32's exponent range; no scaling.
// The DFT_16 matrix is the dense "DFT(16)" block of Table I multiplied as a
// matrix (the paper computes its factors as dense products, Sec. VI).  The
// stage twiddles stay FP32 on the CUDA cores and are applied before the split.
//
// Data flow per CTA is that of the FP32 single-pass kernel: the first stage
// reads HBM, stages exchange through padded shared memory, the last stage
// writes HBM.  The mma fragment layout is produced directly by the loads: the
// lane with groupID g and thread-in-group c loads elements q = 2c, 2c+1,
// 2c+8, 2c+9 of column g, exactly its B-fragment rows, and receives outputs
// m = g, g+8 of columns 2c, 2c+1 in its accumulators.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "stockham.cuh"

namespace gbfft {

enum TcPrec : int { kTcFp16 = 0, kTcBf16 = 1 };

template <int PREC>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if constexpr (PREC == kTcFp16) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// Split two floats into packed (hi, lo) half-type pairs; element 0 in the low
// half.  hi = RN(x) with one packed conversion, lo = RN(x - hi) where x - hi
// is exact in FP32.
template <int PREC>
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    if constexpr (PREC == kTcFp16) {
        const __half2 H = __floats2half2_rn(x0, x1);
        const float2 h = __half22float2(H);
        const __half2 L = __floats2half2_rn(x0 - h.x, x1 - h.y);
        hi = *reinterpret_cast<const uint32_t*>(&H);
        lo = *reinterpret_cast<const uint32_t*>(&L);
    } else {
        const __nv_bfloat162 H = __floats2bfloat162_rn(x0, x1);
        const float2 h = __bfloat1622float2(H);
        const __nv_bfloat162 L = __floats2bfloat162_rn(x0 - h.x, x1 - h.y);
        hi = *reinterpret_cast<const uint32_t*>(&H);
        lo = *reinterpret_cast<const uint32_t*>(&L);
    }
}

// Shared-memory layout of exchange X (after stage X): an XOR swizzle of the
// tile element index that only rewrites bits 0-3 (the 8-byte bank slot) from
// bits >= 4, so it is a bijection on the tile.  It makes the mma-fragment
// reads of the next stage (lanes differ in element bits 0-1 and in the bits of
// q*N/16) and the accumulator writes of this stage (lanes differ in the bits
// of m*L and of the column) land on 16 distinct slots per half-warp.
template <int X>
__device__ __forceinline__ int tc_swz(int i) {
    if constexpr (X == 0) {
        return i ^ (((i >> 5) & 3) << 2) ^ (((i >> 9) & 3) << 2);
    } else {
        return i ^ ((i >> 4) & 1) ^ (((i >> 5) & 1) << 3) ^ (((i >> 9) & 3) << 2);
    }
}

// Exchange index of the stage with this L: 1 -> 0, 16 -> 1, 256 -> 2.
template <int L>
constexpr int tc_stage_index() {
    return L == 1 ? 0 : (L == 16 ? 1 : 2);
}

// A-fragments of M for this lane: frag[(mt*2 + kt)*4 + r] (hi) and +16 (lo).
struct TcFrags {
    uint32_t h[16], l[16];
};

// One radix-16 stage on tensor cores.  FIRST: operands from HBM rows;
// LAST: results to HBM rows; otherwise shared memory in and out.  TPB threads
// cover the stage's T*N/16 columns in tiles of 8 columns per warp.
template <int N, int S, int PREC, int T, int TPB, int PS, int L, bool FIRST, bool LAST>
__device__ __forceinline__ void tc_stage(const ContigIO<N>& io, float2* sm, const float2* __restrict__ tw,
                                         const TcFrags& F, int nvalid) {
    constexpr int R = 16, NR = N / R;
    constexpr int WARPS = TPB / 32;
    constexpr int TILES = T * NR / 8;  // 8-column tiles in the CTA
    constexpr int PER = TILES / WARPS;
    static_assert(TILES % WARPS == 0 && PER >= 1, "tiles split evenly over warps");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, c = lane & 3;
    float2 outv[PER][4];
#pragma unroll
    for (int it = 0; it < PER; ++it) {
        const int tile = warp + it * WARPS;
        // ---- this lane's four elements q = 2c, 2c+1, 2c+8, 2c+9 of column g, twiddled in FP32
        const int B = tile * 8 + g;
        const int t = B / NR, j = B % NR, k = j % L;
        float2 x[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int q = 2 * c + (i & 1) + (i >> 1) * 8;
            const int n = j + q * NR;
            if constexpr (FIRST) {
                x[i] = (t < nvalid) ? io.ld(t, n) : make_float2(0.f, 0.f);
            } else {
                x[i] = sm[tc_swz<tc_stage_index<L>() - 1>(t * N + n)];
            }
            if constexpr (L > 1) {
                if (q > 0) x[i] = twiddle<S>(x[i], __ldg(&tw[(q - 1) * L + k]));
            }
        }
        // ---- per-column power-of-two scale (FP16 only)
        float inv_sc = 1.f;
        if constexpr (PREC == kTcFp16) {
            float m = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) m = fmaxf(m, fmaxf(fabsf(x[i].x), fabsf(x[i].y)));
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
            int e = (int)((__float_as_uint(m) >> 23) & 0xff) - 127;  // floor(log2 m) for normal m
            if (!(m > 0.f)) e = 0;
            e = max(-100, min(100, e));
            const float sc = __uint_as_float((uint32_t)(127 + 14 - e) << 23);
            inv_sc = __uint_as_float((uint32_t)(127 - 14 + e) << 23);
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = make_float2(x[i].x * sc, x[i].y * sc);
        }
        // ---- B fragments: k-tile 0 = real parts, k-tile 1 = imaginary parts
        uint32_t bh[2][2], bl[2][2];
        split2<PREC>(x[0].x, x[1].x, bh[0][0], bl[0][0]);
        split2<PREC>(x[2].x, x[3].x, bh[0][1], bl[0][1]);
        split2<PREC>(x[0].y, x[1].y, bh[1][0], bl[1][0]);
        split2<PREC>(x[2].y, x[3].y, bh[1][1], bl[1][1]);
        // ---- D = Mh Xh + Mh Xl + Ml Xh over 2 x 2 tiles (small terms first)
        float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) {
                const int f = (mt * 2 + kt) * 4;
                const uint32_t ah[4] = {F.h[f], F.h[f + 1], F.h[f + 2], F.h[f + 3]};
                const uint32_t al[4] = {F.l[f], F.l[f + 1], F.l[f + 2], F.l[f + 3]};
                mma16816<PREC>(d[mt], ah, bl[kt][0], bl[kt][1]);
                mma16816<PREC>(d[mt], al, bh[kt][0], bh[kt][1]);
            }
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) {
                const int f = (mt * 2 + kt) * 4;
                const uint32_t ah[4] = {F.h[f], F.h[f + 1], F.h[f + 2], F.h[f + 3]};
                mma16816<PREC>(d[mt], ah, bh[kt][0], bh[kt][1]);
            }
        }
        // ---- outputs: rows g, g+8 of columns 2c, 2c+1; undo those columns' scales
        float s0 = 1.f, s1 = 1.f;
        if constexpr (PREC == kTcFp16) {
            s0 = __shfl_sync(0xffffffffu, inv_sc, (2 * c) * 4);
            s1 = __shfl_sync(0xffffffffu, inv_sc, (2 * c + 1) * 4);
        }
        outv[it][0] = make_float2(d[0][0] * s0, d[1][0] * s0);  // (m = g,   column 2c)
        outv[it][1] = make_float2(d[0][1] * s1, d[1][1] * s1);  // (m = g,   column 2c+1)
        outv[it][2] = make_float2(d[0][2] * s0, d[1][2] * s0);  // (m = g+8, column 2c)
        outv[it][3] = make_float2(d[0][3] * s1, d[1][3] * s1);  // (m = g+8, column 2c+1)
    }
    if constexpr (!FIRST && !LAST) __syncthreads();  // all columns of this stage have been read
#pragma unroll
    for (int it = 0; it < PER; ++it) {
        const int tile = warp + it * WARPS;
        if constexpr (LAST && NR % 2 == 0) {
            // NR even: columns 2c, 2c+1 are adjacent elements j, j+1 (j even) of
            // one output row, so each m is one aligned 16-byte store.
            const int B = tile * 8 + 2 * c;
            const int t = B / NR, j = B % NR;
            if (t < nvalid) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int m = g + 8 * h;
                    float4* dst = reinterpret_cast<float4*>(io.out + t * N + m * L + j);
                    *dst = make_float4(outv[it][2 * h].x, outv[it][2 * h].y, outv[it][2 * h + 1].x,
                                       outv[it][2 * h + 1].y);
                }
            }
        } else {
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int B = tile * 8 + 2 * c + (o & 1);
                const int m = (o < 2) ? g : g + 8;
                const int t = B / NR, j = B % NR;
                const int b = j / L, k = j % L;
                const int n = b * L * R + m * L + k;
                if constexpr (LAST) {
                    if (t < nvalid) io.st(t, n, outv[it][o]);
                } else {
                    sm[tc_swz<tc_stage_index<L>()>(t * N + n)] = outv[it][o];
                }
            }
        }
    }
    if constexpr (!LAST) __syncthreads();
}

// Stages L = 1, 16, 256, ... of the all-radix-16 schedule.  The stage-twiddle
// block of the stage with L >= 16 starts at 15*(16 + ... + L/16) = L - 16.
template <int N, int S, int PREC, int T, int TPB, int PS, int L>
__device__ __forceinline__ void tc_stages(const ContigIO<N>& io, float2* sm, const float2* __restrict__ tw,
                                          const TcFrags& F, int nvalid) {
    constexpr bool LAST = (L * 16 == N);
    tc_stage<N, S, PREC, T, TPB, PS, L, L == 1, LAST>(io, sm, tw + (L > 1 ? L - 16 : 0), F, nvalid);
    if constexpr (!LAST) tc_stages<N, S, PREC, T, TPB, PS, L * 16>(io, sm, tw, F, nvalid);
}

// frag: per lane, 16 hi words then 16 lo words (see k_tc_fragments).
// Persistent: each CTA keeps the DFT_16 fragments in registers and walks the
// tiles blockIdx.x, blockIdx.x + gridDim.x, ...
template <int N, int S, int PREC, int T, int TPB, int PS>
__global__ void __launch_bounds__(TPB) k_stockham_tc(const float2* in, float2* out, const float2* __restrict__ tw,
                                                     const uint32_t* __restrict__ frag, long long batch) {
    extern __shared__ float2 sm[];
    const int lane = threadIdx.x & 31;
    TcFrags F;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        F.h[r] = __ldg(&frag[lane * 32 + r]);
        F.l[r] = __ldg(&frag[lane * 32 + 16 + r]);
    }
    const long long ntiles = (batch + T - 1) / T;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (tile != blockIdx.x) __syncthreads();  // the previous tile's last shared-memory reads are done
        const int nvalid = tile_rows(tile, T, batch);
        const ContigIO<N> io{in + tile * T * N, out + tile * T * N};
        tc_stages<N, S, PREC, T, TPB, PS, 1>(io, sm, tw, F, nvalid);
    }
}

// A-fragment table of M = [[Fr, -Fi], [Fi, Fr]] (DFT_16 over the reals) for
// mma.m16n8k16 row-major A: for lane (g, c) and tile (mt, kt), register r
// holds rows g + 8*(r & 1), columns 2c + 8*(r >> 1) + {0, 1} of the tile.
// Entries are evaluated in FP64 (sincospi of the exactly reduced angle) and
// split as hi = RN(x), lo = RN(x - hi) in the half type.
__global__ void k_tc_fragments(uint32_t* frag, int prec, int sign) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // lane*32 + part*16 + tile*4 + r, one word
    if (idx >= 32 * 32) return;
    const int lane = idx / 32, rest = idx % 32;
    const int part = rest / 16, tile = (rest % 16) / 4, r = rest % 4;
    const int mt = tile / 2, kt = tile % 2;
    const int g = lane >> 2, c = lane & 3;
    const int row = g + 8 * (r & 1);
    uint32_t word = 0;
    for (int h = 0; h < 2; ++h) {
        const int col = 2 * c + 8 * (r >> 1) + h;
        const int e = (row * col) % 16;
        double sn, cs;
        sincospi(2.0 * (double)e / 16.0, &sn, &cs);
        const double fr = cs, fi = (double)sign * sn;  // F = exp(sign * 2 pi i m q / 16)
        double v;
        if (mt == 0 && kt == 0) v = fr;
        else if (mt == 0 && kt == 1) v = -fi;
        else if (mt == 1 && kt == 0) v = fi;
        else v = fr;
        uint16_t bits;
        if (prec == kTcFp16) {
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
        word |= (uint32_t)bits << (16 * h);
    }
    frag[idx] = word;
}

cudaError_t launch_tc_fragments(uint32_t* frag, int prec, int sign, cudaStream_t s) {
    k_tc_fragments<<<4, 256, 0, s>>>(frag, prec, sign);
    return cudaGetLastError();
}

template <int N, int T, int TPB, int PS>
inline TcVariant make_tc_variant() {
    static_assert(((T * (N / 16) / 8) % (TPB / 32)) == 0, "tiles split evenly over warps");
    int nst = 0;
    for (int m = N; m > 1; m /= 16) ++nst;
    TcVariant v{};
    v.n = N;
    v.rows = T;
    v.tpb = TPB;
    v.nstages = nst;
    v.smem = nst > 1 ? (int)(T * N * sizeof(float2)) : 0;
    v.k[0][0] = (const void*)&k_stockham_tc<N, -1, kTcFp16, T, TPB, PS>;
    v.k[0][1] = (const void*)&k_stockham_tc<N, +1, kTcFp16, T, TPB, PS>;
    v.k[1][0] = (const void*)&k_stockham_tc<N, -1, kTcBf16, T, TPB, PS>;
    v.k[1][1] = (const void*)&k_stockham_tc<N, +1, kTcBf16, T, TPB, PS>;
    return v;
}

static const TcVariant kTc[] = {
    make_tc_variant<16, 64, 128, 0>(),
    make_tc_variant<256, 8, 128, 4>(),
    make_tc_variant<4096, 1, 256, 4>(),
};

const TcVariant* tc_variant_for(int64_t n) {
    for (const TcVariant& v : kTc)
        if (v.n == n) return &v;
    return nullptr;
}

int tc_grid(const TcVariant& v) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.k[0][0], v.tpb, (size_t)v.smem) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

cudaError_t launch_tc(const TcVariant& v, int prec, int direction, const float2* in, float2* out, const float2* tw,
                      const uint32_t* frag, long long batch, int grid_cap, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    long long blocks = (batch + v.rows - 1) / v.rows;
    if (grid_cap > 0 && blocks > grid_cap) blocks = grid_cap;
    void* args[] = {(void*)&in, (void*)&out, (void*)&tw, (void*)&frag, (void*)&batch};
    const void* fn = v.k[prec][direction == GBFFT_FORWARD ? 0 : 1];
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(v.tpb), args, (size_t)v.smem, s);
}

cudaError_t prepare_tc(const TcVariant& v) {
    if (v.smem <= 48 * 1024) return cudaSuccess;
    for (int p = 0; p < 2; ++p)
        for (int d = 0; d < 2; ++d) {
            cudaError_t e = cudaFuncSetAttribute(v.k[p][d], cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

}  // namespace gbfft
