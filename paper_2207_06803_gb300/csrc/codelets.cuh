// Register codelets: DFT_r for r in {2, 3, 4, 5, 7, 8, 16, 32, 64}, fully unrolled.
//
// Each codelet computes A = DFT_r a in place on r complex values held in
// registers, natural order in and out, with DFT_r[m][k] = w^(m*k) and
// w = exp(S * 2*pi*i / r) (S = -1 forward, Sec. II; S = +1 inverse).  These
// are the "DFT(r)" generators of Table I evaluated as straight-line code, the
// GPU counterpart of the small solved sub-problems a DFT planner bottoms out in
// (Sec. III).  Composite codelets use the split of Eq. 2 internally
// (DFT_8 = 2 x 4, DFT_16 = 4 x 4, DFT_32 = 2 x 16, DFT_64 = 8 x 8); the odd primes use the symmetric
// sum/difference form of the direct DFT.
#pragma once
#include <cuda_runtime.h>

namespace gbfft {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// a * (S * i)
template <int S>
__device__ __forceinline__ float2 mul_si(float2 a) {
    return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// a * (c + i*S*s) for compile-time constants c, s
template <int S>
__device__ __forceinline__ float2 mul_const(float2 a, float c, float s) {
    const float ss = S > 0 ? s : -s;
    return make_float2(fmaf(a.x, c, -a.y * ss), fmaf(a.x, ss, a.y * c));
}
// Twiddle application for direction S from a forward-table entry w = exp(-2*pi*i*e/N).
template <int S>
__device__ __forceinline__ float2 twiddle(float2 a, float2 w) {
    return S < 0 ? cmul(a, w) : cmulc(a, w);
}

constexpr float kC8 = 0.70710678118654752440f;   // cos(pi/4)
constexpr float kC16 = 0.92387953251128675613f;  // cos(pi/8)
constexpr float kS16 = 0.38268343236508977173f;  // sin(pi/8)

template <int S, int R>
struct Dft;

template <int S>
struct Dft<S, 2> {
    __device__ __forceinline__ static void run(float2* a) {
        float2 t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    }
};

template <int S>
struct Dft<S, 4> {
    __device__ __forceinline__ static void run(float2* a) {
        float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
        float2 t2 = cadd(a[1], a[3]), t3 = mul_si<S>(csub(a[1], a[3]));
        a[0] = cadd(t0, t2);
        a[2] = csub(t0, t2);
        a[1] = cadd(t1, t3);
        a[3] = csub(t1, t3);
    }
};

// DFT_8: even/odd split (K = 2, M = 4 in Eq. 2).
template <int S>
struct Dft<S, 8> {
    __device__ __forceinline__ static void run(float2* a) {
        float2 e[4] = {a[0], a[2], a[4], a[6]};
        float2 o[4] = {a[1], a[3], a[5], a[7]};
        Dft<S, 4>::run(e);
        Dft<S, 4>::run(o);
        o[1] = mul_const<S>(o[1], kC8, kC8);    // w8^1
        o[2] = mul_si<S>(o[2]);                 // w8^2
        o[3] = mul_const<S>(o[3], -kC8, kC8);   // w8^3
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a[k] = cadd(e[k], o[k]);
            a[k + 4] = csub(e[k], o[k]);
        }
    }
};

// DFT_16 as 4 x 4 (K = M = 4 in Eq. 2):
//   X[j1 + 4*j2] = sum_k w4^(j2*k) * w16^(j1*k) * sum_m w4^(j1*m) x[4m + k].
template <int S>
struct Dft<S, 16> {
    __device__ __forceinline__ static void run(float2* a) {
        float2 z[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int m = 0; m < 4; ++m) z[k][m] = a[4 * m + k];
            Dft<S, 4>::run(z[k]);
        }
        // w16^(j1*k) for j1, k in 1..3: exponents 1, 2, 3, 4, 6, 9
        z[1][1] = mul_const<S>(z[1][1], kC16, kS16);
        z[1][2] = mul_const<S>(z[1][2], kC8, kC8);
        z[1][3] = mul_const<S>(z[1][3], kS16, kC16);
        z[2][1] = mul_const<S>(z[2][1], kC8, kC8);
        z[2][2] = mul_si<S>(z[2][2]);
        z[2][3] = mul_const<S>(z[2][3], -kC8, kC8);
        z[3][1] = mul_const<S>(z[3][1], kS16, kC16);
        z[3][2] = mul_const<S>(z[3][2], -kC8, kC8);
        z[3][3] = mul_const<S>(z[3][3], -kC16, -kS16);
#pragma unroll
        for (int j1 = 0; j1 < 4; ++j1) {
            float2 c[4] = {z[0][j1], z[1][j1], z[2][j1], z[3][j1]};
            Dft<S, 4>::run(c);
#pragma unroll
            for (int j2 = 0; j2 < 4; ++j2) a[j1 + 4 * j2] = c[j2];
        }
    }
};

// cos(pi*j/16), j = 0..8 (sin(pi*j/16) = cos(pi*(8-j)/16)).
__device__ __forceinline__ constexpr float cos_pi16(int j) {
    return j == 0 ? 1.0f
         : j == 1 ? 0.98078528040323044913f
         : j == 2 ? 0.92387953251128675613f
         : j == 3 ? 0.83146961230254523708f
         : j == 4 ? 0.70710678118654752440f
         : j == 5 ? 0.55557023301960222474f
         : j == 6 ? 0.38268343236508977173f
         : j == 7 ? 0.19509032201612826785f
                  : 0.0f;
}

// a * w32^j for j in 0..15, w32 = exp(S*2*pi*i/32) = (cos(pi j/16), S sin(pi j/16)).
template <int S>
__device__ __forceinline__ float2 mul_w32(float2 a, int j) {
    if (j == 0) return a;
    if (j == 8) return mul_si<S>(a);
    const float c = j < 8 ? cos_pi16(j) : -cos_pi16(16 - j);
    const float s = j < 8 ? cos_pi16(8 - j) : cos_pi16(j - 8);
    return mul_const<S>(a, c, s);
}

// DFT_32: even/odd split (K = 2, M = 16 in Eq. 2).
template <int S>
struct Dft<S, 32> {
    __device__ __forceinline__ static void run(float2* a) {
        float2 e[16], o[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            e[m] = a[2 * m];
            o[m] = a[2 * m + 1];
        }
        Dft<S, 16>::run(e);
        Dft<S, 16>::run(o);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float2 t = mul_w32<S>(o[k], k);
            a[k] = cadd(e[k], t);
            a[k + 16] = csub(e[k], t);
        }
    }
};

// cos(pi*j/32), j = 0..16.
__device__ __forceinline__ constexpr float cos_pi32(int j) {
    return j == 0 ? 1.0f
         : j == 1 ? 0.99518472667219688624f
         : j == 2 ? 0.98078528040323044913f
         : j == 3 ? 0.95694033573220886494f
         : j == 4 ? 0.92387953251128675613f
         : j == 5 ? 0.88192126434835502971f
         : j == 6 ? 0.83146961230254523708f
         : j == 7 ? 0.77301045336273696081f
         : j == 8 ? 0.70710678118654752440f
         : j == 9 ? 0.63439328416364549822f
         : j == 10 ? 0.55557023301960222474f
         : j == 11 ? 0.47139673682599764856f
         : j == 12 ? 0.38268343236508977173f
         : j == 13 ? 0.29028467725446236764f
         : j == 14 ? 0.19509032201612826785f
         : j == 15 ? 0.09801714032956060199f
                   : 0.0f;
}

// a * w64^e for 0 <= e < 64, w64 = exp(S*2*pi*i/64) = (cos(pi e/32), S sin(pi e/32)),
// with the angle reduced to the first octant by quadrant symmetry.
template <int S>
__device__ __forceinline__ float2 mul_w64(float2 a, int e) {
    e &= 63;
    if (e == 0) return a;
    if (e == 16) return mul_si<S>(a);
    if (e == 32) return make_float2(-a.x, -a.y);
    if (e == 48) return mul_si<-S>(a);
    float c, s;
    if (e < 16) {
        c = cos_pi32(e);
        s = cos_pi32(16 - e);
    } else if (e < 32) {
        c = -cos_pi32(32 - e);
        s = cos_pi32(e - 16);
    } else if (e < 48) {
        c = -cos_pi32(e - 32);
        s = -cos_pi32(48 - e);
    } else {
        c = cos_pi32(64 - e);
        s = -cos_pi32(e - 48);
    }
    return mul_const<S>(a, c, s);
}

// DFT_64 as 8 x 8 (K = M = 8 in Eq. 2):
//   X[j1 + 8*j2] = sum_k w8^(j2*k) * w64^(j1*k) * sum_m w8^(j1*m) x[8m + k].
template <int S>
struct Dft<S, 64> {
    __device__ __forceinline__ static void run(float2* a) {
        float2 z[8][8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
#pragma unroll
            for (int m = 0; m < 8; ++m) z[k][m] = a[8 * m + k];
            Dft<S, 8>::run(z[k]);
#pragma unroll
            for (int j1 = 1; j1 < 8; ++j1) z[k][j1] = mul_w64<S>(z[k][j1], j1 * k);
        }
#pragma unroll
        for (int j1 = 0; j1 < 8; ++j1) {
            float2 c[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) c[k] = z[k][j1];
            Dft<S, 8>::run(c);
#pragma unroll
            for (int j2 = 0; j2 < 8; ++j2) a[j1 + 8 * j2] = c[j2];
        }
    }
};

// Odd prime p: with t_m = a_m + a_{p-m}, u_m = a_m - a_{p-m} (m = 1..h, h = (p-1)/2),
//   A_k     = a_0 + sum_m cos(2 pi k m / p) t_m + i*S * sum_m sin(2 pi k m / p) u_m
//   A_{p-k} = a_0 + sum_m cos(2 pi k m / p) t_m - i*S * sum_m sin(2 pi k m / p) u_m.
template <int P>
struct PrimeConsts;
template <>
struct PrimeConsts<3> {
    __device__ __forceinline__ static float c(int j) { return -0.5f; }
    __device__ __forceinline__ static float s(int j) { return 0.86602540378443864676f; }
};
template <>
struct PrimeConsts<5> {
    __device__ __forceinline__ static float c(int j) {
        return j == 1 ? 0.30901699437494742410f : -0.80901699437494742410f;
    }
    __device__ __forceinline__ static float s(int j) {
        return j == 1 ? 0.95105651629515357212f : 0.58778525229247312917f;
    }
};
template <>
struct PrimeConsts<7> {
    __device__ __forceinline__ static float c(int j) {
        return j == 1 ? 0.62348980185873353053f : (j == 2 ? -0.22252093395631440429f : -0.90096886790241912624f);
    }
    __device__ __forceinline__ static float s(int j) {
        return j == 1 ? 0.78183148246802980871f : (j == 2 ? 0.97492791218182360702f : 0.43388373911755812048f);
    }
};

template <int S, int P>
struct DftPrime {
    __device__ __forceinline__ static void run(float2* a) {
        constexpr int H = (P - 1) / 2;
        float2 t[H + 1], u[H + 1];
#pragma unroll
        for (int m = 1; m <= H; ++m) {
            t[m] = cadd(a[m], a[P - m]);
            u[m] = csub(a[m], a[P - m]);
        }
        float2 a0 = a[0];
        float2 sum = a0;
#pragma unroll
        for (int m = 1; m <= H; ++m) sum = cadd(sum, t[m]);
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            float2 pr = a0, qs = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 1; m <= H; ++m) {
                // (k*m mod P) folded onto 1..H: cos is even, sin is odd.
                const int e = (k * m) % P;
                const int f = e <= H ? e : P - e;
                const float cs = PrimeConsts<P>::c(f);
                const float sn = e <= H ? PrimeConsts<P>::s(f) : -PrimeConsts<P>::s(f);
                pr.x = fmaf(cs, t[m].x, pr.x);
                pr.y = fmaf(cs, t[m].y, pr.y);
                qs.x = fmaf(sn, u[m].x, qs.x);
                qs.y = fmaf(sn, u[m].y, qs.y);
            }
            const float2 iq = mul_si<S>(qs);  // i*S*Q
            a[k] = cadd(pr, iq);
            a[P - k] = csub(pr, iq);
        }
        a[0] = sum;
    }
};

template <int S>
struct Dft<S, 3> : DftPrime<S, 3> {};
template <int S>
struct Dft<S, 5> : DftPrime<S, 5> {};
template <int S>
struct Dft<S, 7> : DftPrime<S, 7> {};

}  // namespace gbfft
