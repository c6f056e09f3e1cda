// Register codelets: DFT_r for r in {2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 20, 24, 28, 32, 40, 48, 56, 64}, fully unrolled, on
// float2 (FP32 path) or double2 (FP64 path) values.
//
// Each codelet computes A = DFT_r a in place on r complex values held in
// registers, natural order in and out, with DFT_r[m][k] = w^(m*k) and
// w = exp(S * 2*pi*i / r) (S = -1 forward, Sec. II; S = +1 inverse).  These
// are the "DFT(r)" generators of Table I evaluated as straight-line code, the
// GPU counterpart of the small solved sub-problems a DFT planner bottoms out in
// (Sec. III).  Composite codelets use the split of Eq. 2 internally
// (DFT_8 = 2 x 4, DFT_16 = 4 x 4, DFT_32 = 2 x 16, DFT_64 = 8 x 8); the odd primes use the symmetric
// sum/difference form of the direct DFT; the products of an odd prime and a power of two
// (6, 10, 12, 14, 20, 24, 28, 40, 48, 56) use the prime-factor map, which needs no twiddles.
#pragma once
#include <cuda_runtime.h>

namespace gbfft {

// Complex values are C (FP32 path) or double2 (FP64 path); every helper
// below exists for both, and the codelets are templates over the type.
template <class C>
struct RealOf;
template <>
struct RealOf<float2> {
    using T = float;
};
template <>
struct RealOf<double2> {
    using T = double;
};

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

template <class C>
__device__ __forceinline__ C cadd(C a, C b) {
    return C{a.x + b.x, a.y + b.y};
}
template <class C>
__device__ __forceinline__ C csub(C a, C b) {
    return C{a.x - b.x, a.y - b.y};
}
template <class C>
__device__ __forceinline__ C cmul(C a, C b) {
    return C{fmaT(a.x, b.x, -a.y * b.y), fmaT(a.x, b.y, a.y * b.x)};
}
// a * conj(b)
template <class C>
__device__ __forceinline__ C cmulc(C a, C b) {
    return C{fmaT(a.x, b.x, a.y * b.y), fmaT(a.y, b.x, -a.x * b.y)};
}
// a * (S * i)
template <int S, class C>
__device__ __forceinline__ C mul_si(C a) {
    return S > 0 ? C{-a.y, a.x} : C{a.y, -a.x};
}
// a * (c + i*S*s) for compile-time constants c, s (given in double precision
// and rounded once to the working precision).
template <int S, class C>
__device__ __forceinline__ C mul_const(C a, double cd, double sd) {
    using T = typename RealOf<C>::T;
    const T c = (T)cd, s = (T)sd;
    const T ss = S > 0 ? s : -s;
    return C{fmaT(a.x, c, -a.y * ss), fmaT(a.x, ss, a.y * c)};
}
// Twiddle application for direction S from a forward-table entry w = exp(-2*pi*i*e/N).
template <int S, class C>
__device__ __forceinline__ C twiddle(C a, C w) {
    return S < 0 ? cmul(a, w) : cmulc(a, w);
}

constexpr double kC8 = 0.70710678118654752440;   // cos(pi/4)
constexpr double kC16 = 0.92387953251128675613;  // cos(pi/8)
constexpr double kS16 = 0.38268343236508977173;  // sin(pi/8)

template <int S, int R>
struct Dft;

template <int S>
struct Dft<S, 2> {
    template <class C>
    __device__ __forceinline__ static void run(C* a) {
        C t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    }
};

template <int S>
struct Dft<S, 4> {
    template <class C>
    __device__ __forceinline__ static void run(C* a) {
        C t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
        C t2 = cadd(a[1], a[3]), t3 = mul_si<S>(csub(a[1], a[3]));
        a[0] = cadd(t0, t2);
        a[2] = csub(t0, t2);
        a[1] = cadd(t1, t3);
        a[3] = csub(t1, t3);
    }
};

// DFT_8: even/odd split (K = 2, M = 4 in Eq. 2).
template <int S>
struct Dft<S, 8> {
    template <class C>
    __device__ __forceinline__ static void run(C* a) {
        C e[4] = {a[0], a[2], a[4], a[6]};
        C o[4] = {a[1], a[3], a[5], a[7]};
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
    template <class C>
    __device__ __forceinline__ static void run(C* a) {
        C z[4][4];
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
            C c[4] = {z[0][j1], z[1][j1], z[2][j1], z[3][j1]};
            Dft<S, 4>::run(c);
#pragma unroll
            for (int j2 = 0; j2 < 4; ++j2) a[j1 + 4 * j2] = c[j2];
        }
    }
};

// cos(pi*j/16), j = 0..8 (sin(pi*j/16) = cos(pi*(8-j)/16)).
__device__ __forceinline__ constexpr double cos_pi16(int j) {
    return j == 0 ? 1.0
         : j == 1 ? 0.98078528040323044913
         : j == 2 ? 0.92387953251128675613
         : j == 3 ? 0.83146961230254523708
         : j == 4 ? 0.70710678118654752440
         : j == 5 ? 0.55557023301960222474
         : j == 6 ? 0.38268343236508977173
         : j == 7 ? 0.19509032201612826785
                  : 0.0;
}

// a * w32^j for j in 0..15, w32 = exp(S*2*pi*i/32) = (cos(pi j/16), S sin(pi j/16)).
template <int S, class C>
__device__ __forceinline__ C mul_w32(C a, int j) {
    if (j == 0) return a;
    if (j == 8) return mul_si<S>(a);
    const double c = j < 8 ? cos_pi16(j) : -cos_pi16(16 - j);
    const double s = j < 8 ? cos_pi16(8 - j) : cos_pi16(j - 8);
    return mul_const<S>(a, c, s);
}

// DFT_32: even/odd split (K = 2, M = 16 in Eq. 2).
template <int S>
struct Dft<S, 32> {
    template <class C>
    __device__ __forceinline__ static void run(C* a) {
        C e[16], o[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            e[m] = a[2 * m];
            o[m] = a[2 * m + 1];
        }
        Dft<S, 16>::run(e);
        Dft<S, 16>::run(o);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const C t = mul_w32<S>(o[k], k);
            a[k] = cadd(e[k], t);
            a[k + 16] = csub(e[k], t);
        }
    }
};

// cos(pi*j/32), j = 0..16.
__device__ __forceinline__ constexpr double cos_pi32(int j) {
    return j == 0 ? 1.0
         : j == 1 ? 0.99518472667219688624
         : j == 2 ? 0.98078528040323044913
         : j == 3 ? 0.95694033573220886494
         : j == 4 ? 0.92387953251128675613
         : j == 5 ? 0.88192126434835502971
         : j == 6 ? 0.83146961230254523708
         : j == 7 ? 0.77301045336273696081
         : j == 8 ? 0.70710678118654752440
         : j == 9 ? 0.63439328416364549822
         : j == 10 ? 0.55557023301960222474
         : j == 11 ? 0.47139673682599764856
         : j == 12 ? 0.38268343236508977173
         : j == 13 ? 0.29028467725446236764
         : j == 14 ? 0.19509032201612826785
         : j == 15 ? 0.09801714032956060199
                   : 0.0;
}

// a * w64^e for 0 <= e < 64, w64 = exp(S*2*pi*i/64) = (cos(pi e/32), S sin(pi e/32)),
// with the angle reduced to the first octant by quadrant symmetry.
template <int S, class C>
__device__ __forceinline__ C mul_w64(C a, int e) {
    e &= 63;
    if (e == 0) return a;
    if (e == 16) return mul_si<S>(a);
    if (e == 32) return C{-a.x, -a.y};
    if (e == 48) return mul_si<-S>(a);
    double c, s;
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
    template <class C>
    __device__ __forceinline__ static void run(C* a) {
        C z[8][8];
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
            C c[8];
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
    __device__ __forceinline__ static double c(int j) { return -0.5; }
    __device__ __forceinline__ static double s(int j) { return 0.86602540378443864676; }
};
template <>
struct PrimeConsts<5> {
    __device__ __forceinline__ static double c(int j) {
        return j == 1 ? 0.30901699437494742410 : -0.80901699437494742410;
    }
    __device__ __forceinline__ static double s(int j) {
        return j == 1 ? 0.95105651629515357212 : 0.58778525229247312917;
    }
};
template <>
struct PrimeConsts<7> {
    __device__ __forceinline__ static double c(int j) {
        return j == 1 ? 0.62348980185873353053 : (j == 2 ? -0.22252093395631440429 : -0.90096886790241912624);
    }
    __device__ __forceinline__ static double s(int j) {
        return j == 1 ? 0.78183148246802980871 : (j == 2 ? 0.97492791218182360702 : 0.43388373911755812048);
    }
};

template <int S, int P>
struct DftPrime {
    template <class C>
    __device__ __forceinline__ static void run(C* a) {
        constexpr int H = (P - 1) / 2;
        C t[H + 1], u[H + 1];
#pragma unroll
        for (int m = 1; m <= H; ++m) {
            t[m] = cadd(a[m], a[P - m]);
            u[m] = csub(a[m], a[P - m]);
        }
        C a0 = a[0];
        C sum = a0;
#pragma unroll
        for (int m = 1; m <= H; ++m) sum = cadd(sum, t[m]);
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            C pr = a0, qs = C{};
#pragma unroll
            for (int m = 1; m <= H; ++m) {
                // (k*m mod P) folded onto 1..H: cos is even, sin is odd.
                const int e = (k * m) % P;
                const int f = e <= H ? e : P - e;
                using T = typename RealOf<C>::T;
                const T cs = (T)PrimeConsts<P>::c(f);
                const T sn = (T)(e <= H ? PrimeConsts<P>::s(f) : -PrimeConsts<P>::s(f));
                pr.x = fmaT(cs, t[m].x, pr.x);
                pr.y = fmaT(cs, t[m].y, pr.y);
                qs.x = fmaT(sn, u[m].x, qs.x);
                qs.y = fmaT(sn, u[m].y, qs.y);
            }
            const C iq = mul_si<S>(qs);  // i*S*Q
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

// x^-1 mod m for coprime x, m (compile time).
constexpr int inverse_mod(int x, int m) {
    for (int y = 0; y < m; ++y)
        if ((x * y) % m == 1 % m) return y;
    return -1;
}

// DFT_{P*Q} for coprime P, Q by the prime-factor (Good-Thomas) index maps:
// input n = (Q*n1 + P*n2) mod PQ, output k with k = k1 (mod P), k = k2 (mod Q)
// (k = (k1*Q*(Q^-1 mod P) + k2*P*(P^-1 mod Q)) mod PQ, the Chinese remainder
// map).  Then w_PQ^(nk) = w_P^(n1*k1) * w_Q^(n2*k2), so
//   A_k = sum_n1 w_P^(n1 k1) sum_n2 w_Q^(n2 k2) a[(Q n1 + P n2) mod PQ]:
// P DFT_Q over n2, then Q DFT_P over n1, with no twiddle factors between them
// (unlike the split of Eq. 2, which needs them when the factors share a
// divisor).  All indices are compile-time constants: the maps cost no
// instructions.
template <int S, int P, int Q>
struct DftPfa {
    template <class C>
    __device__ __forceinline__ static void run(C* a) {
        constexpr int R = P * Q;
        constexpr int QI = inverse_mod(Q % P, P), PI = inverse_mod(P % Q, Q);
        static_assert(QI >= 0 && PI >= 0, "P and Q must be coprime");
        C y[P][Q];
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) {
#pragma unroll
            for (int n2 = 0; n2 < Q; ++n2) y[n1][n2] = a[(Q * n1 + P * n2) % R];
            Dft<S, Q>::run(y[n1]);
        }
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) {
            C z[P];
#pragma unroll
            for (int n1 = 0; n1 < P; ++n1) z[n1] = y[n1][k2];
            Dft<S, P>::run(z);
#pragma unroll
            for (int k1 = 0; k1 < P; ++k1) a[(k1 * Q * QI + k2 * P * PI) % R] = z[k1];
        }
    }
};

template <int S>
struct Dft<S, 6> : DftPfa<S, 3, 2> {};
template <int S>
struct Dft<S, 10> : DftPfa<S, 5, 2> {};
template <int S>
struct Dft<S, 12> : DftPfa<S, 3, 4> {};
template <int S>
struct Dft<S, 14> : DftPfa<S, 7, 2> {};
template <int S>
struct Dft<S, 20> : DftPfa<S, 5, 4> {};
template <int S>
struct Dft<S, 24> : DftPfa<S, 3, 8> {};
template <int S>
struct Dft<S, 28> : DftPfa<S, 7, 4> {};
template <int S>
struct Dft<S, 40> : DftPfa<S, 5, 8> {};
template <int S>
struct Dft<S, 48> : DftPfa<S, 3, 16> {};
template <int S>
struct Dft<S, 56> : DftPfa<S, 7, 8> {};

}  // namespace gbfft
