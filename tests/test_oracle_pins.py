"""Pins for the CPU FP64 oracle, checked against what the paper and the
mathematics fix rather than against the oracle itself:

* the worked examples the paper prints (Eq. 1's factor matrices, Listing 1's
  4-point program), stored under ``tests/golden/``;
* closed forms of the DFT of Sec. II for special inputs (delta, constant,
  complex tone, real cosine, geometric sequence), which a dropped term, a sign
  flip, an index slip or a transposed operand would break;
* invariants (linearity, shift theorem, Parseval, inverse(forward(x)) = N x);
* the Eq. 2 factorisation rebuilt densely with np.kron for small (K, M);
* cross-checks between the oracle's three independent transforms and, as a
  third opinion (the paper's own correctness check, Sec. VI), numpy.fft.

Run on CPU; no GPU needed.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FWD, INV = oracle.FORWARD, oracle.INVERSE

POW2 = [1, 2, 4, 8, 16, 32, 64, 128, 256, 1024, 4096]
MIXED = [3, 5, 6, 7, 9, 10, 12, 14, 15, 21, 25, 35, 49, 60, 105, 210, 384, 640, 896]
TRANSFORMS = {
    "naive": oracle.dft_naive,
    "radix2": oracle.fft_radix2,
    "eq2": oracle.fft_eq2,
}


def sizes_for(kind):
    if kind == "radix2":
        return POW2
    return POW2 + MIXED


def rel_err(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def rng_complex(n, batch=1, seed=0):
    r = np.random.default_rng(seed)
    return r.standard_normal((batch, n)) + 1j * r.standard_normal((batch, n))


# --------------------------------------------------------------------------
# Worked examples printed in the paper
# --------------------------------------------------------------------------

def load_listing1():
    rows = []
    with open(os.path.join(GOLDEN, "listing1_dft4.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(v) for v in line.split()])
    a = np.array(rows)
    return a[:, 1] + 1j * a[:, 2], a[:, 3] + 1j * a[:, 4]


def load_eq1():
    mats, name = {}, None
    with open(os.path.join(GOLDEN, "eq1_dft4_factors.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            if line.startswith("matrix"):
                name = line.split()[1]
                mats[name] = []
                continue
            row = []
            for tok in line.split():
                re, im = tok.split(",")
                row.append((int(re), int(im)))
            mats[name].append(row)
    return mats


def gauss_matmul(a, b):
    """Exact product of matrices of Gaussian integers given as (re, im) pairs."""
    n, k, m = len(a), len(b), len(b[0])
    out = [[(0, 0)] * m for _ in range(n)]
    for i in range(n):
        for j in range(m):
            re = im = 0
            for t in range(k):
                ar, ai = a[i][t]
                br, bi = b[t][j]
                re += ar * br - ai * bi
                im += ar * bi + ai * br
            out[i][j] = (re, im)
    return out


def test_eq1_printed_factors_multiply_to_dft4_exactly():
    m = load_eq1()
    prod = gauss_matmul(m["DFT2_kron_I2"], gauss_matmul(
        m["twiddle_diag"], gauss_matmul(m["I2_kron_DFT2"], m["stride_permutation"])))
    assert prod == m["DFT4"]


@pytest.mark.parametrize("kind", list(TRANSFORMS))
def test_oracle_matrix_at_n4_is_eq1_dft4(kind):
    dft4 = np.array([[complex(*e) for e in row] for row in load_eq1()["DFT4"]])
    cols = TRANSFORMS[kind](np.eye(4, dtype=np.complex128), FWD)  # row k = DFT_4 e_k
    assert np.max(np.abs(cols.T - dft4)) < 1e-15


@pytest.mark.parametrize("kind", list(TRANSFORMS))
def test_listing1_program_output(kind):
    x, y = load_listing1()
    out = TRANSFORMS[kind](x, FWD)
    assert np.max(np.abs(out - y)) < 1e-13


def test_dft3_closed_form():
    # DFT_3 with omega = exp(-2 pi i / 3) = -1/2 - i sqrt(3)/2.
    w = complex(-0.5, -math.sqrt(3.0) / 2.0)
    mat = np.array([[1, 1, 1], [1, w, w * w], [1, w * w, w]])
    for kind in ("naive", "eq2"):
        cols = TRANSFORMS[kind](np.eye(3, dtype=np.complex128), FWD)
        assert np.max(np.abs(cols.T - mat)) < 1e-15


def test_dft2_closed_form():
    for kind in TRANSFORMS:
        cols = TRANSFORMS[kind](np.eye(2, dtype=np.complex128), FWD)
        assert np.max(np.abs(cols.T - np.array([[1, 1], [1, -1]]))) < 1e-15


# --------------------------------------------------------------------------
# Closed forms of the DFT for special inputs
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", list(TRANSFORMS))
@pytest.mark.parametrize("sign", [FWD, INV])
def test_delta_gives_all_ones(kind, sign):
    for n in sizes_for(kind):
        x = np.zeros(n, complex)
        x[0] = 1
        assert np.max(np.abs(TRANSFORMS[kind](x, sign) - 1)) < 1e-14, n


@pytest.mark.parametrize("kind", list(TRANSFORMS))
@pytest.mark.parametrize("sign", [FWD, INV])
def test_constant_gives_scaled_delta(kind, sign):
    c = 0.75 - 1.25j
    for n in sizes_for(kind):
        y = TRANSFORMS[kind](np.full(n, c), sign)
        want = np.zeros(n, complex)
        want[0] = n * c
        assert np.max(np.abs(y - want)) < 1e-12 * n, n


@pytest.mark.parametrize("kind", list(TRANSFORMS))
def test_complex_tone_lands_in_one_bin(kind):
    # Forward (omega = exp(-2 pi i/N)): sum_k exp(+2 pi i f k/N) omega^(m k) = N [m == f].
    # The inverse maps exp(-2 pi i f k / N) to N [m == f].  Either sign error
    # moves the peak to bin N - f.
    for n in sizes_for(kind):
        if n < 3:
            continue
        f = (3 * n) // 7 or 1
        k = np.arange(n)
        want = np.zeros(n, complex)
        want[f] = n
        for sign in (FWD, INV):
            x = np.exp(-sign * 2j * np.pi * f * k / n)
            assert np.max(np.abs(TRANSFORMS[kind](x, sign) - want)) < 1e-11 * n, (n, sign)


@pytest.mark.parametrize("kind", list(TRANSFORMS))
def test_real_cosine_gives_two_bins(kind):
    for n in sizes_for(kind):
        if n < 5:
            continue
        f = n // 5
        x = np.cos(2 * np.pi * f * np.arange(n) / n).astype(complex)
        want = np.zeros(n, complex)
        want[f] += n / 2
        want[n - f] += n / 2
        assert np.max(np.abs(TRANSFORMS[kind](x, FWD) - want)) < 1e-11 * n, n


@pytest.mark.parametrize("kind", list(TRANSFORMS))
@pytest.mark.parametrize("sign", [FWD, INV])
def test_geometric_sequence_closed_form(kind, sign):
    # x[k] = a^k  =>  y[m] = sum_k (a w^m)^k = (1 - a^N) / (1 - a w^m),  w = exp(sign 2 pi i/N).
    a = 0.93 * np.exp(0.37j)
    for n in sizes_for(kind):
        k = np.arange(n)
        x = a ** k
        w_m = np.exp(sign * 2j * np.pi * k / n)
        want = (1 - a ** n) / (1 - a * w_m)
        assert rel_err(TRANSFORMS[kind](x, sign), want) < 1e-13, n


@pytest.mark.parametrize("kind", list(TRANSFORMS))
def test_shifted_delta_is_a_column_of_powers(kind):
    # delta at s: y[m] = omega^(m s); checked through the recurrence y[m+1] = y[m] * omega^s
    # and y[0] = 1, which does not evaluate the closed form term by term.
    for n in sizes_for(kind):
        if n < 2:
            continue
        s = n // 3 + 1 if n > 3 else 1
        x = np.zeros(n, complex)
        x[s % n] = 1
        y = TRANSFORMS[kind](x, FWD)
        step = np.exp(-2j * np.pi * (s % n) / n)
        assert abs(y[0] - 1) < 1e-14
        assert np.max(np.abs(y[1:] - y[:-1] * step)) < 1e-12, n


# --------------------------------------------------------------------------
# Invariants of the DFT
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", list(TRANSFORMS))
def test_linearity(kind):
    for n in sizes_for(kind):
        x, z = rng_complex(n, 2, seed=n)
        a, b = 1.5 - 0.5j, -0.25 + 2j
        f = TRANSFORMS[kind]
        assert rel_err(f(a * x + b * z), a * f(x) + b * f(z)) < 1e-13, n


@pytest.mark.parametrize("kind", list(TRANSFORMS))
def test_shift_theorem(kind):
    for n in sizes_for(kind):
        if n < 2:
            continue
        x = rng_complex(n, 1, seed=7 * n)[0]
        s = (2 * n) // 5 or 1
        y = TRANSFORMS[kind](x, FWD)
        ys = TRANSFORMS[kind](np.roll(x, s), FWD)  # x[k - s]
        m = np.arange(n)
        assert rel_err(ys, y * np.exp(-2j * np.pi * ((m * s) % n) / n)) < 1e-13, n


@pytest.mark.parametrize("kind", list(TRANSFORMS))
def test_parseval(kind):
    for n in sizes_for(kind):
        x = rng_complex(n, 3, seed=11 * n)
        y = TRANSFORMS[kind](x, FWD)
        lhs = np.sum(np.abs(y) ** 2, axis=1)
        rhs = n * np.sum(np.abs(x) ** 2, axis=1)
        assert np.max(np.abs(lhs - rhs) / rhs) < 1e-13, n


@pytest.mark.parametrize("kind", list(TRANSFORMS))
def test_inverse_of_forward_is_n_times_x(kind):
    for n in sizes_for(kind):
        x = rng_complex(n, 2, seed=13 * n)
        f = TRANSFORMS[kind]
        assert rel_err(f(f(x, FWD), INV), n * x) < 1e-13, n


# --------------------------------------------------------------------------
# Eq. 2 as a dense matrix identity (readings of D^N_M and Pi^N_K)
# --------------------------------------------------------------------------

def dense_dft(n):
    return oracle.dft_naive(np.eye(n, dtype=np.complex128), FWD).T


def twiddle_diag(n, m):
    k_blocks = n // m
    d = np.array([np.exp(-2j * np.pi * (k * j % n) / n) for k in range(k_blocks) for j in range(m)])
    return np.diag(d)


def stride_perm(n, k_blocks):
    m = n // k_blocks
    p = np.zeros((n, n))
    for k in range(k_blocks):
        for j in range(m):
            p[k * m + j, j * k_blocks + k] = 1
    return p


@pytest.mark.parametrize("k_blocks,m", [(2, 2), (2, 3), (3, 2), (3, 5), (7, 4), (5, 2), (4, 4), (2, 8)])
def test_eq2_factorisation_dense(k_blocks, m):
    n = k_blocks * m
    rhs = (np.kron(dense_dft(k_blocks), np.eye(m)) @ twiddle_diag(n, m)
           @ np.kron(np.eye(k_blocks), dense_dft(m)) @ stride_perm(n, k_blocks))
    assert np.max(np.abs(rhs - dense_dft(n))) < 1e-13


def test_eq2_readings_reproduce_eq1():
    m = load_eq1()
    to = lambda mat: np.array([[complex(*e) for e in row] for row in mat])
    assert np.allclose(twiddle_diag(4, 2), to(m["twiddle_diag"]), atol=1e-15)
    assert np.array_equal(stride_perm(4, 2), to(m["stride_permutation"]).real)


# --------------------------------------------------------------------------
# Cross-checks between independent implementations
# --------------------------------------------------------------------------

@pytest.mark.parametrize("sign", [FWD, INV])
def test_three_transforms_agree(sign):
    for n in POW2:
        x = rng_complex(n, 4, seed=n)
        a = oracle.dft_naive(x, sign)
        assert rel_err(oracle.fft_radix2(x, sign), a) < 1e-13, n
        assert rel_err(oracle.fft_eq2(x, sign), a) < 1e-13, n
    for n in MIXED:
        x = rng_complex(n, 4, seed=n)
        assert rel_err(oracle.fft_eq2(x, sign), oracle.dft_naive(x, sign)) < 1e-13, n


def test_ragged_family_sizes_eq2_vs_naive():
    from paper_2207_06803_gb300 import synth
    fam = synth.size_family(8, 8192)
    assert len(fam) == 41
    for n in fam:
        x = rng_complex(n, 1, seed=n)
        assert rel_err(oracle.fft_eq2(x), oracle.dft_naive(x)) < 1e-13, n


def test_large_sizes_eq2_vs_radix2():
    for n in (8192, 16384):
        x = rng_complex(n, 2, seed=n)
        assert rel_err(oracle.fft_eq2(x), oracle.fft_radix2(x)) < 1e-13, n


def test_numpy_fft_third_opinion():
    # Sec. VI checks against NumPy's FFT; here it is only a third opinion.
    for n in POW2 + MIXED:
        x = rng_complex(n, 2, seed=3 * n)
        assert rel_err(oracle.fft_eq2(x, FWD), np.fft.fft(x, axis=1)) < 1e-13, n
        assert rel_err(oracle.fft_eq2(x, INV), n * np.fft.ifft(x, axis=1)) < 1e-13, n


def test_threaded_matches_single_thread():
    x = rng_complex(64, 37, seed=5)
    for f in TRANSFORMS.values():
        assert np.array_equal(f(x, FWD, nthreads=1), f(x, FWD, nthreads=4))


def test_invalid_arguments_rejected():
    with pytest.raises(ValueError):
        oracle.fft_radix2(np.zeros(12, complex))


def direct_nd(x, sign):
    """The multi-dimensional DFT by its definition: one sum over every index
    tuple, y[k] = sum_n x[n] exp(sign 2 pi i sum_a k_a n_a / d_a)."""
    import itertools
    dims = x.shape
    out = np.zeros(dims, np.complex128)
    for k in itertools.product(*[range(d) for d in dims]):
        acc = 0j
        for n in itertools.product(*[range(d) for d in dims]):
            phase = sum(ki * ni / d for ki, ni, d in zip(k, n, dims))
            acc += x[n] * np.exp(sign * 2j * np.pi * phase)
        out[k] = acc
    return out


@pytest.mark.parametrize("dims", [(3, 4), (2, 5), (2, 3, 4), (4, 1, 3)])
@pytest.mark.parametrize("sign", [FWD, INV])
def test_dft_nd_is_the_multidimensional_definition(dims, sign):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(dims) + 1j * rng.standard_normal(dims)
    got = oracle.dft_nd(x[None], sign)[0]
    assert np.max(np.abs(got - direct_nd(x, sign))) < 1e-12 * math.prod(dims)


def test_dft_nd_planted_mistakes_fail_the_definition():
    """Plausible slips in an axis-by-axis multi-dimensional DFT (an axis
    skipped, one axis transformed with the opposite sign, the axes' lengths
    swapped on a non-square shape) each disagree with the direct sum."""
    dims = (3, 4)
    rng = np.random.default_rng(11)
    x = rng.standard_normal(dims) + 1j * rng.standard_normal(dims)
    want = direct_nd(x, FWD)
    skipped = oracle.dft(x, FWD)                                  # last axis only
    wrong_sign = oracle.dft(oracle.dft(x.T, INV).T, FWD)          # axis 0 inverse
    swapped = oracle.dft(oracle.dft(x.reshape(4, 3), FWD).T, FWD).T.reshape(dims)
    for bad in (skipped, wrong_sign, swapped):
        assert np.max(np.abs(bad - want)) > 1e-3
    right = oracle.dft(oracle.dft(x, FWD).T, FWD).T
    assert np.max(np.abs(right - want)) < 1e-12
