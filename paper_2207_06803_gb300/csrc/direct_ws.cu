// Direct DFT on the tensor cores, warp-specialised and pipelined (the
// paper's "direct DFT", Sec. VI: y = F_N x as one dense product, no
// factorisation).  The arithmetic is that of direct.cu: per tile of 128
// transforms, D = A B^T with A = [xr xi] (128 x 2N, one transform per row,
// split into high and low half-precision parts, FP16 rows first scaled by an
// exact power of two) and B = [Bh; Bl] the real form of F_N, so that
// D = Al Bh^T + Ah Bl^T + Ah Bh^T accumulates in FP32 in tensor memory.
//
// What differs is the schedule.  direct.cu runs load, split, MMA, read-back
// and store of a tile one after the other in every thread of a CTA; here
// three roles run concurrently on consecutive tiles, handing tiles over
// through two tensor-memory slots (each: D, Ah, Al of one tile) and mbarriers:
//   producers  (warps 0-3, warp q owns rows 32q .. 32q+31 of a tile = TMEM
//              lanes 32q ..): coalesced 16-byte loads of the warp's 32 rows
//              (contiguous in HBM) into its shared staging rows, then each
//              lane splits its own row into Ah / Al and stores them into its
//              TMEM lane (tcgen05.st) -- A never touches shared memory;
//              arrive on full[slot];
//   MMA        (warp 8, one thread): waits full[slot], issues the 3 * 2N/16
//              MMAs with A read from tensor memory and B resident in shared
//              memory, commits to done[slot];
//   epilogue   (warps 4-7, warp 4+q reads TMEM lanes 32q ..): waits
//              done[slot], reads its lanes' rows of D (tcgen05.ld), scales,
//              arrives on free[slot] (the slot may take the tile after next),
//              then writes the rows through its shared staging rows with
//              coalesced 16-byte stores.
// The producer of tile i+2 waits free[slot]; the MMA of tile i waits full,
// so D of a slot is overwritten only after its rows were read.  Every wait is
// bounded (globaltimer deadline) and its outcome made uniform across the warp;
// on expiry the kernel records GBFFT_ERR_TIMEOUT, lets the other roles run out
// their own bounded waits, waits for its last MMAs, frees its tensor memory
// and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "internal.h"
#include "tcgen05.cuh"

namespace gbfft {
namespace {

constexpr unsigned long long kWsWaitNs = 1000000000ull;
constexpr int kWsRows = 128;      // transforms per tile (the MMA's M)
constexpr int kWsThreads = 288;   // producers 0-3, epilogue 4-7, MMA 8
constexpr int kWsSmemMax = 232448 - 1024;  // dynamic shared memory per CTA (227 KB less the CTA's reservation)
constexpr int kEpiChunk = 8;      // complex per epilogue chunk (8 measured faster than 16)
constexpr int kEpiPitch = 8 * kEpiChunk + 16;  // epilogue staging: one chunk of a row, padded

constexpr uint32_t ws_cols(int c) { return c <= 32 ? 32u : (c <= 64 ? 64u : (c <= 128 ? 128u : (c <= 256 ? 256u : 512u))); }
constexpr int ws_min(int a, int b) { return a < b ? a : b; }

template <int N>
struct WsGeom {
    static constexpr int K = 2 * N;                 // [re parts | im parts]
    static constexpr int SBO = 16 * K;              // B: 8-row groups of K/8 core matrices
    static constexpr int B_BYTES = 2 * K * K * 2;   // [Bh; Bl]
    static constexpr int PITCH = 8 * N + 16;        // producer staging row pitch (bytes): conflict-free row reads
    static constexpr int STAGE = 32 * PITCH;        // one warp's 32 rows of one tile
    static constexpr int SLOT = 4 * N;              // TMEM columns per slot: D 2N, Ah N, Al N
    static constexpr int NSLOT = ws_min(4, 512 / SLOT);
    static constexpr uint32_t COLS = ws_cols(NSLOT * SLOT);
    static constexpr int OFF_RING = (B_BYTES + 1023) / 1024 * 1024;
    static constexpr int EPI = 4 * 32 * kEpiPitch;
    static constexpr int FIXED = OFF_RING + EPI + NSLOT * kWsRows * 4 + 3 * NSLOT * 8 + 16;
    // staging tiles per producer warp: as many as fit, at most 12 (N <= 16) or 6
    static constexpr int NSTG = ws_min(N <= 16 ? 12 : 6, (kWsSmemMax - FIXED) / (4 * STAGE));
    // Tiles beyond the staged ones whose rows are also requested into L2 (bulk prefetch): one for the
    // lengths 24, 40, 56 (24: 5.79 -> 6.44 TB/s, 40: 5.78 -> 6.45, 56: 6.03 -> 6.36), none for the
    // others, which a prefetch slowed (64: 5.92 -> 5.71, 16: 6.22 -> 5.90, 8: 5.47 -> 4.56).
    static constexpr int PREFETCH = N % 16 == 8 && N > 8 ? 1 : 0;
    static constexpr int OFF_EPI = OFF_RING + 4 * NSTG * STAGE;
    static constexpr int OFF_EXP = OFF_EPI + EPI;
    static constexpr int OFF_BAR = OFF_EXP + NSLOT * kWsRows * 4;
    static constexpr int SMEM = OFF_BAR + 3 * NSLOT * 8 + 16;
    static_assert(N % 8 == 0 && K <= 256 && NSLOT >= 2 && NSTG >= 2 && SMEM <= kWsSmemMax,
                  "direct DFT: N a multiple of 8 up to 64");
};

// Bounded mbarrier wait whose outcome every lane of the warp shares.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, kWsWaitNs) ? 1 : 0) != 0;
}

// 16-byte asynchronous copy global -> shared; zero-fills when !valid (src then unread).
__device__ __forceinline__ void cp16(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// Bulk prefetch of `bytes` (a multiple of 16, from a 16-byte-aligned address) into L2.
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

template <int N, int S, int PREC>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_dft_direct_ws(const float2* in, float2* out, const uint4* __restrict__ bmat, long long batch, int* status) {
    using G = WsGeom<N>;
    constexpr int K = G::K, F4 = N / 2, CPR = N / 8;  // float4 (2 complex) and 8-complex chunks per row
    constexpr int NP = F4;                            // float4 per lane when a warp moves its 32 rows
    constexpr int NSLOT = G::NSLOT, NSTG = G::NSTG;
    extern __shared__ __align__(1024) uint8_t dsm[];
    uint8_t* const bsm = dsm;
    uint8_t* const ring = dsm + G::OFF_RING;
    uint8_t* const epi = dsm + G::OFF_EPI;
    int* const s_exp = reinterpret_cast<int*>(dsm + G::OFF_EXP);
    uint64_t* const full = reinterpret_cast<uint64_t*>(dsm + G::OFF_BAR);  // [NSLOT]: producers -> MMA
    uint64_t* const done = full + NSLOT;                                   // [NSLOT]: MMA -> epilogue
    uint64_t* const free_ = full + 2 * NSLOT;                              // [NSLOT]: epilogue -> producers
    uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(full + 3 * NSLOT);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < G::B_BYTES / 16; i += kWsThreads) reinterpret_cast<uint4*>(bsm)[i] = bmat[i];
    if (tid == 0) {
        for (int s = 0; s < NSLOT; ++s) {
            mbar_init(&full[s], 4);
            mbar_init(&done[s], 1);
            mbar_init(&free_[s], 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(G::COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async_smem();  // B, written by ordinary stores, is read by the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const long long ntiles = (batch + kWsRows - 1) / kWsRows;
    // This CTA's tiles: first, first + stride, ... below last (every gridDim-th tile; contiguous runs
    // of tiles per CTA measured slower, N = 40: 6.31 -> 5.74 TB/s).
    const long long first = blockIdx.x, last = ntiles, stride = gridDim.x;
    bool ok = true;
    if (warp < 4) {  // producers
        const int q = warp;
        uint8_t* const mine = ring + q * NSTG * G::STAGE;  // this warp's ring of staging tiles
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        // The warp's 32 rows of `tile` (contiguous in HBM) into staging tile b with coalesced 16-byte
        // asynchronous copies (rows past the batch read as zeros); one copy group per call.
        auto issue = [&](long long tile, int b) {
            if (G::PREFETCH > 0 && lane == 0) {  // the warp's rows of a later tile into L2, one bulk request
                const long long pt = tile + G::PREFETCH * stride;
                const long long p0 = pt * kWsRows + q * 32;
                const long long pn = max(0LL, min(32LL, batch - p0));
                if (pt < last && pn > 0) prefetch_l2(in + p0 * N, (uint32_t)(pn * N * 8));
            }
            if (tile < last) {
                const long long r0 = tile * kWsRows + q * 32;
                const int nv = (int)max(0LL, min(32LL, batch - r0));
                const float4* src = reinterpret_cast<const float4*>(in + r0 * N);
                uint8_t* const dst = mine + b * G::STAGE;
#pragma unroll
                for (int e = 0; e < NP; ++e) {
                    const int p = lane + 32 * e, row = p / F4, c = p - row * F4;
                    const bool valid = row < nv;
                    cp16(dst + row * G::PITCH + c * 16, valid ? (const void*)(src + p) : (const void*)in, valid);
                }
            }
            cp_commit();
        };
#pragma unroll 1
        for (int j = 0; j < NSTG; ++j) issue(first + j * stride, j);
        int b = 0, s = 0;
        uint32_t u = 0;  // uses of slot s so far
        long long it = 0;
        for (long long tile = first; tile < last; tile += stride, ++it) {
            cp_wait<NSTG - 1>();  // this lane's copies of tile `it` (the oldest group) have landed
            __syncwarp();         // ... and every lane's
            if (it >= NSLOT && !warp_wait(&free_[s], (u - 1) & 1)) {  // the epilogue has read this slot's D
                ok = false;
                break;
            }
            // lane = row: scale (FP16), split, store Ah / Al into this lane of the slot
            const float4* rowp = reinterpret_cast<const float4*>(mine + b * G::STAGE + lane * G::PITCH);
            float sc = 1.f;
            if constexpr (PREC == 0) {  // exact power-of-two scale of the row to [2^14, 2^15)
                float m = 0.f;
#pragma unroll
                for (int c = 0; c < F4; ++c) {
                    const float4 w = rowp[c];
                    m = fmaxf(m, fmaxf(fmaxf(fabsf(w.x), fabsf(w.y)), fmaxf(fabsf(w.z), fabsf(w.w))));
                }
                int ex = (int)((__float_as_uint(m) >> 23) & 0xff) - 127;
                if (!(m > 0.f)) ex = 0;
                ex = max(-100, min(100, ex));
                s_exp[s * kWsRows + q * 32 + lane] = ex;
                sc = __uint_as_float((uint32_t)(127 + 14 - ex) << 23);
            }
            // K index k of A at column k / 2 (two halves per column): real parts k = n, imaginary k = N + n
            const uint32_t ah = tmem + lane_base + (uint32_t)(s * G::SLOT + 2 * N), al = ah + (uint32_t)N;
#pragma unroll
            for (int c = 0; c < CPR; ++c) {
                uint32_t hr[4], lr[4], hi_[4], li[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const float4 w = rowp[4 * c + p];  // complex 8c + 2p (x, y) and 8c + 2p + 1 (z, w)
                    float a, bb;
                    hr[p] = pack_hi<PREC>(w.x * sc, w.z * sc, a, bb);
                    lr[p] = pack_lo<PREC>(a, bb);
                    hi_[p] = pack_hi<PREC>(w.y * sc, w.w * sc, a, bb);
                    li[p] = pack_lo<PREC>(a, bb);
                }
                tmem_st4(ah + (uint32_t)(4 * c), hr);
                tmem_st4(al + (uint32_t)(4 * c), lr);
                tmem_st4(ah + (uint32_t)(N / 2 + 4 * c), hi_);
                tmem_st4(al + (uint32_t)(N / 2 + 4 * c), li);
            }
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();  // also: every lane is done reading staging tile b
            if (lane == 0) mbar_arrive(&full[s]);
            issue(tile + NSTG * stride, b);  // refill the staging tile just read
            b = b + 1 == NSTG ? 0 : b + 1;
            if (++s == NSLOT) {
                s = 0;
                ++u;
            }
        }
        cp_wait<0>();  // no copy into this CTA's shared memory is left in flight
    } else if (warp < 8) {  // epilogue
        const int q = warp - 4;
        uint8_t* const st = epi + q * 32 * kEpiPitch;  // one 8-complex chunk of each of the warp's 32 rows
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int s = 0;
        uint32_t u = 0;
        for (long long tile = first; tile < last; tile += stride) {
            // D of this tile is complete; waiting on the producers' phase too orders their scale
            // exponents before the reads below (that phase cannot advance before free[s] is arrived)
            if (!warp_wait(&done[s], u & 1) || !warp_wait(&full[s], u & 1)) {
                ok = false;
                break;
            }
            tc_fence_after();
            float inv = 1.f;
            if constexpr (PREC == 0)
                inv = __uint_as_float((uint32_t)(127 - 14 + s_exp[s * kWsRows + q * 32 + lane]) << 23);
            const uint32_t d = tmem + lane_base + (uint32_t)(s * G::SLOT);
            const long long r0 = tile * kWsRows + q * 32;
            const int nv = (int)max(0LL, min(32LL, batch - r0));
            float4* dst = reinterpret_cast<float4*>(out + r0 * N);
            float4* srow = reinterpret_cast<float4*>(st + lane * kEpiPitch);
            // Columns [c0, c0 + CW) of the real and the imaginary parts: both loads in flight before one
            // wait, then the chunk of the warp's 32 rows (CW * 8 contiguous bytes per row) leaves through
            // the staging rows, CW / 2 lanes per row.
            auto chunk = [&](int c0, auto cw) {
                constexpr int CW = decltype(cw)::value;
                uint32_t rr[CW], ri[CW];
                if constexpr (CW == 16) {
                    tmem_ld16_nw(d + (uint32_t)c0, rr);
                    tmem_ld16_nw(d + (uint32_t)(N + c0), ri);
                } else {
                    tmem_ld8_nw(d + (uint32_t)c0, rr);
                    tmem_ld8_nw(d + (uint32_t)(N + c0), ri);
                }
                tmem_ld_wait();
#pragma unroll
                for (int h = 0; h < CW / 2; ++h)
                    srow[h] = make_float4(__uint_as_float(rr[2 * h]) * inv, __uint_as_float(ri[2 * h]) * inv,
                                          __uint_as_float(rr[2 * h + 1]) * inv, __uint_as_float(ri[2 * h + 1]) * inv);
                __syncwarp();
                constexpr int PPR = CW / 2;  // 16-byte pieces per row of the chunk
#pragma unroll
                for (int k = 0; k < PPR; ++k) {
                    const int p = lane + 32 * k, row = p / PPR, h = p % PPR;
                    if (row < nv)
                        dst[row * F4 + c0 / 2 + h] = *reinterpret_cast<const float4*>(st + row * kEpiPitch + h * 16);
                }
                __syncwarp();
            };
            if constexpr (kEpiChunk == 16) {
#pragma unroll
                for (int c0 = 0; c0 + 16 <= N; c0 += 16) chunk(c0, std::integral_constant<int, 16>());
                if constexpr (N % 16 == 8) chunk(N - 8, std::integral_constant<int, 8>());
            } else {
#pragma unroll
                for (int c0 = 0; c0 < N; c0 += 8) chunk(c0, std::integral_constant<int, 8>());
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&free_[s]);  // every read of this slot's D is done
            if (++s == NSLOT) {
                s = 0;
                ++u;
            }
        }
    } else {  // warp 8: one thread issues the MMAs
        if (lane == 0) {
            const uint32_t idesc = tc_instr_desc(PREC, kWsRows, K);
            const uint32_t bh = smem_u32(bsm), bl = bh + (uint32_t)(K / 8) * G::SBO;  // rows K..2K-1 = Bl
            int s = 0, last_s = -1;
            uint32_t u = 0, last_u = 0;
            for (long long tile = first; tile < last; tile += stride) {
                if (!mbar_wait(&full[s], u & 1, kWsWaitNs)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(s * G::SLOT), ah = d + 2 * N, al = d + 3 * N;
                // D = Al Bh^T + Ah Bl^T + Ah Bh^T (small terms first), K = 16 per instruction
#pragma unroll
                for (int ks = 0; ks < K / 16; ++ks)
                    tc_mma_f16_ta(d, al + (uint32_t)(ks * 8), tc_smem_desc(bh + ks * 256, 128, G::SBO), idesc, ks);
#pragma unroll
                for (int ks = 0; ks < K / 16; ++ks)
                    tc_mma_f16_ta(d, ah + (uint32_t)(ks * 8), tc_smem_desc(bl + ks * 256, 128, G::SBO), idesc, 1);
#pragma unroll
                for (int ks = 0; ks < K / 16; ++ks)
                    tc_mma_f16_ta(d, ah + (uint32_t)(ks * 8), tc_smem_desc(bh + ks * 256, 128, G::SBO), idesc, 1);
                tc_commit(&done[s]);
                last_s = s;
                last_u = u;
                if (++s == NSLOT) {
                    s = 0;
                    ++u;
                }
            }
            // the tensor memory is freed below: the last MMAs issued must have completed
            if (last_s >= 0 && !mbar_wait(&done[last_s], last_u & 1, kWsWaitNs)) ok = false;
        }
        __syncwarp();
    }
    if (!ok) atomicCAS(status, 0, (int)GBFFT_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 8)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::COLS) : "memory");
}

template <int N>
DirectWsVariant make_ws_variant() {
    DirectWsVariant v{};
    v.n = N;
    v.tpb = kWsThreads;
    v.smem = WsGeom<N>::SMEM;
    v.tmem_cols = (int)WsGeom<N>::COLS;
    v.k[0][0] = (const void*)&k_dft_direct_ws<N, -1, 0>;
    v.k[0][1] = (const void*)&k_dft_direct_ws<N, +1, 0>;
    v.k[1][0] = (const void*)&k_dft_direct_ws<N, -1, 1>;
    v.k[1][1] = (const void*)&k_dft_direct_ws<N, +1, 1>;
    return v;
}

const DirectWsVariant kDirectWs[] = {
    make_ws_variant<8>(),  make_ws_variant<16>(), make_ws_variant<24>(), make_ws_variant<32>(),
    make_ws_variant<40>(), make_ws_variant<48>(), make_ws_variant<56>(), make_ws_variant<64>(),
};

}  // namespace

const DirectWsVariant* direct_ws_variant_for(int64_t n) {
    for (const DirectWsVariant& v : kDirectWs)
        if (v.n == n) return &v;
    return nullptr;
}

cudaError_t prepare_direct_ws(const DirectWsVariant& v) {
    for (int p = 0; p < 2; ++p)
        for (int d = 0; d < 2; ++d) {
            const cudaError_t e = cudaFuncSetAttribute(v.k[p][d], cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

// Resident CTAs per SM (occupancy of the kernel and its tensor-memory
// columns, 512 per SM), times the SM count.
int direct_ws_grid(const DirectWsVariant& v) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.k[0][0], v.tpb, (size_t)v.smem) != cudaSuccess)
        return 0;
    per_sm = std::min(per_sm, 512 / v.tmem_cols);
    return per_sm < 1 ? 0 : per_sm * sms;
}

cudaError_t launch_direct_ws(const DirectWsVariant& v, int prec, int direction, const float2* in, float2* out,
                             const void* bmat, long long batch, int grid_cap, int* status, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    long long blocks = (batch + kWsRows - 1) / kWsRows;
    if (grid_cap > 0 && blocks > grid_cap) blocks = grid_cap;
    void* args[] = {(void*)&in, (void*)&out, (void*)&bmat, (void*)&batch, (void*)&status};
    const void* fn = v.k[prec][direction == GBFFT_FORWARD ? 0 : 1];
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(v.tpb), args, (size_t)v.smem, s);
}

}  // namespace gbfft
