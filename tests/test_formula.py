"""Factorisation-formula front end (Table I vocabulary, Eq. 2): the host-side
checker through the C ABI against a dense evaluation of the same formulas
(written here from Table I's operator meanings and Eq. 2's readings of D and
Pi), syntax handling, and formula-driven plans on the GPU."""
import math

import numpy as np
import pytest

from paper_2207_06803_gb300 import gbfft, synth

KRON, DOT = "⊗", "·"   # the paper's operator symbols


# -- formulas as small trees, rendered to text and evaluated densely ---------

def dft(n):
    return ("DFT", n)


def eye(n):
    return ("I", n)


def tw(n, m):
    return ("twiddle", n, m)


def perm(n, k):
    return ("Permute", n, k)


def kron(a, b):
    return ("kron", a, b)


def prod(*fs):
    return ("prod",) + tuple(fs)


def size(f):
    if f[0] in ("DFT", "I", "twiddle", "Permute"):
        return f[1]
    if f[0] == "kron":
        return size(f[1]) * size(f[2])
    return size(f[1])


def eq2(outer, inner):
    """Eq. 2 with DFT factors `outer` (size K) and `inner` (size M)."""
    k, m = size(outer), size(inner)
    n = k * m
    return prod(kron(outer, eye(m)), tw(n, m), kron(eye(k), inner), perm(n, k))


def eq2_transposed(outer, inner):
    """The transpose of Eq. 2 (decimation in frequency): DFT_K runs first, then DFT_M."""
    k, m = size(outer), size(inner)
    n = k * m
    return prod(perm(n, m), kron(eye(k), inner), tw(n, m), kron(outer, eye(m)))


def ct(radices):
    """Recursive Cooley-Tukey formula whose DFT leaves, in application order, are `radices`."""
    if len(radices) == 1:
        return dft(radices[0])
    return eq2(dft(radices[-1]), ct(radices[:-1]))


def reversal(n, r):
    """Base-r digit reversal of length n: Rev_n = (I_r (x) Rev_(n/r)) . Permute(n, r), Rev_r = I_r."""
    if n == r:
        return eye(r)
    return prod(kron(eye(r), reversal(n // r, r)), perm(n, r))


def pease(r, t, short=False):
    """Pease's constant-geometry product G_t ... G_1 Rev_N for N = r^t, with
    G_s = (DFT_r (x) I_(N/r)) . (twiddle(r^s, r^(s-1)) (x) I(r^(t-s))) . Permute(N, r);
    `short` writes G_t's twiddle without its I(1) and Rev_(r^2) as Permute(r^2, r)."""
    n = r ** t
    fs = []
    for s in range(t, 0, -1):
        twf = tw(r ** s, r ** (s - 1))
        if not (short and s == t):
            twf = kron(twf, eye(r ** (t - s)))
        fs += [kron(dft(r), eye(n // r)), twf, perm(n, r)]
    rev = reversal(n, r)
    if short and t == 2:
        rev = perm(n, r)
    fs += list(rev[1:]) if rev[0] == "prod" else [rev]
    return prod(*fs)


def render(f, ascii_ops=False):
    k_op = " kron " if ascii_ops else f" {KRON} "
    d_op = " * " if ascii_ops else f" {DOT} "
    if f[0] in ("DFT", "I"):
        return f"{f[0]}({f[1]})"
    if f[0] in ("twiddle", "Permute"):
        return f"{f[0]}({f[1]},{f[2]})"
    if f[0] == "kron":
        return "(" + render(f[1], ascii_ops) + k_op + render(f[2], ascii_ops) + ")"
    return "(" + d_op.join(render(g, ascii_ops) for g in f[1:]) + ")"


def dense(f):
    """The matrix a formula denotes (Table I; D^N_M = diag(w_N^(k j)) at k*M + j,
    (Pi^N_K x)[k*M + m] = x[m*K + k]), in FP64."""
    if f[0] == "DFT":
        n = f[1]
        idx = np.arange(n)
        return np.exp(-2j * np.pi * np.outer(idx, idx) / n)
    if f[0] == "I":
        return np.eye(f[1], dtype=complex)
    if f[0] == "twiddle":
        n, m = f[1], f[2]
        k = np.arange(n) // m
        j = np.arange(n) % m
        return np.diag(np.exp(-2j * np.pi * ((k * j) % n) / n))
    if f[0] == "Permute":
        n, kb = f[1], f[2]
        m = n // kb
        p = np.zeros((n, n), dtype=complex)
        for k in range(kb):
            for mm in range(m):
                p[k * m + mm, mm * kb + k] = 1
        return p
    if f[0] == "kron":
        return np.kron(dense(f[1]), dense(f[2]))
    out = dense(f[1])
    for g in f[2:]:
        out = out @ dense(g)
    return out


def is_dft(f):
    n = size(f)
    return np.allclose(dense(f), dense(dft(n)), atol=1e-9)


def checker_accepts(text):
    try:
        return gbfft.gbfft_formula_check(text)
    except gbfft.GbfftError:
        return None


# -- the checker (host only) -------------------------------------------------

def test_eq1_as_a_formula():
    r = gbfft.gbfft_formula_check(render(eq2(dft(2), dft(2))))
    assert r == {"n": 4, "k_outer": 2, "leaves": [2, 2]}


@pytest.mark.parametrize("radices", [[2, 2], [4, 2], [2, 3], [3, 5, 2], [16, 16], [2, 16, 16], [7, 4, 2],
                                     [8, 8, 8, 8], [2] * 12, [64, 128]])
def test_recursive_formulas(radices):
    f = ct(radices)
    r = gbfft.gbfft_formula_check(render(f))
    assert r["n"] == math.prod(radices) and r["leaves"] == radices and r["k_outer"] == radices[-1]
    assert gbfft.gbfft_formula_check(render(f, ascii_ops=True)) == r


@pytest.mark.parametrize("k,m", [(2, 2), (2, 4), (4, 2), (3, 5), (8, 16)])
def test_transposed_form(k, m):
    f = eq2_transposed(dft(k), dft(m))
    assert is_dft(f) if k * m <= 64 else True
    r = gbfft.gbfft_formula_check(render(f))
    assert r == {"n": k * m, "k_outer": k, "leaves": [k, m]}
    if k != m:  # its mistakes: Eq. 2's permutation argument, or Eq. 2's factor order with these factors
        bad = prod(perm(k * m, k), kron(eye(k), dft(m)), tw(k * m, m), kron(dft(k), eye(m)))
        assert not is_dft(bad) and checker_accepts(render(bad)) is None


def test_mixed_forms_nest():
    f = eq2(eq2_transposed(dft(2), dft(4)), ct([4, 2]))
    assert is_dft(f)
    assert gbfft.gbfft_formula_check(render(f)) == {"n": 64, "k_outer": 8, "leaves": [4, 2, 2, 4]}


def test_split_on_both_factors():
    f = eq2(ct([2, 4]), ct([4, 2]))          # outer DFT_8 and inner DFT_8 both factorised
    r = gbfft.gbfft_formula_check(render(f))
    assert r == {"n": 64, "k_outer": 8, "leaves": [4, 2, 2, 4]}


def mutations(k, m):
    """Plausible mistakes in Eq. 2 for DFT_(k m): each denotes another matrix when k != m."""
    n = k * m
    good = [kron(dft(k), eye(m)), tw(n, m), kron(eye(k), dft(m)), perm(n, k)]
    yield "twiddle arguments swapped", prod(good[0], tw(n, k), good[2], good[3])
    yield "permutation arguments swapped", prod(good[0], good[1], good[2], perm(n, m))
    yield "outer Kronecker factors swapped", prod(kron(eye(m), dft(k)), good[1], good[2], good[3])
    yield "inner Kronecker factors swapped", prod(good[0], good[1], kron(dft(m), eye(k)), good[3])
    yield "twiddle dropped", prod(good[0], good[2], good[3])
    yield "permutation dropped", prod(good[0], good[1], good[2])
    yield "factors reordered", prod(good[0], good[2], good[1], good[3])


@pytest.mark.parametrize("k,m", [(2, 2), (2, 4), (4, 2), (3, 5), (5, 3), (2, 8), (4, 4)])
def test_checker_agrees_with_dense_evaluation(k, m):
    """Pins the checker to the mathematics: it accepts a formula iff the formula
    denotes DFT_N (for Eq. 2 and its plausible mistakes)."""
    good = eq2(dft(k), dft(m))
    assert is_dft(good) and checker_accepts(render(good)) is not None
    for why, f in mutations(k, m):
        if size_ok(f) and is_dft(f):
            continue  # the mistake is invisible at this (k, m), e.g. swapped arguments when k == m
        assert checker_accepts(render(f)) is None, why


def size_ok(f):
    if f[0] == "prod":
        sizes = {size(g) for g in f[1:]}
        return len(sizes) == 1 and all(size_ok(g) for g in f[1:])
    if f[0] == "kron":
        return size_ok(f[1]) and size_ok(f[2])
    return True


@pytest.mark.parametrize("radices", [[2, 2, 2], [3, 2, 2], [4, 3], [2, 5, 3]])
def test_accepted_recursive_formulas_are_dfts_densely(radices):
    f = ct(radices)
    assert checker_accepts(render(f)) is not None and is_dft(f)


def test_program_line_and_input_vector():
    body = render(eq2(dft(4), dft(8)))
    for text in (f"var y = {body} {DOT} x;", f"{body} {DOT} InputComplex", f"var result={body};", body):
        assert gbfft.gbfft_formula_check(text)["n"] == 32
    assert gbfft.gbfft_formula_check("DFT(12)") == {"n": 12, "k_outer": 0, "leaves": [12]}


@pytest.mark.parametrize("text,why", [
    ("DFT(4", "expected ')'"),
    ("DFT(0)", "n >= 1"),
    ("(DFT(2) kron I(2)) * twiddle(4,2) * (I(2) kron DFT(2))", "four factors"),
    ("DFT(2) kron I(2) * twiddle(4,2)", "equal dimensions"),
    ("I(4)", "not a DFT"),
    ("x * DFT(4)", "last factor"),
    ("DFT(4) + DFT(4)", "unexpected text"),
    ("twiddle(4,3)", "divisor"),
    ("", "expected a factor"),
])
def test_rejections_carry_a_reason(text, why):
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_formula_check(text)
    assert e.value.status == gbfft.GBFFT_ERR_INVALID_ARG
    assert why in str(e.value), str(e.value)


# -- Pease's constant-geometry form ------------------------------------------

PEASE_CASES = [(2, 2), (2, 3), (2, 4), (3, 2), (3, 3), (4, 2), (4, 3), (5, 2), (8, 2), (16, 2)]


@pytest.mark.parametrize("r,t", PEASE_CASES)
def test_pease_form_is_dft_densely(r, t):
    """Pins the reading of Pease's factorisation (derived from Eq. 2 with K = r:
    the permutations of the unrolled recursion gathered into one digit reversal
    applied first, each stage G_s with the same geometry) to the DFT matrix by
    dense evaluation, and the checker to the same formulas."""
    for short in (False, True):
        f = pease(r, t, short)
        assert is_dft(f), (r, t, short)
        got = checker_accepts(render(f))
        assert got == {"n": r ** t, "k_outer": 0, "leaves": [r] * t}, (r, t, short, got)
        assert gbfft.gbfft_formula_form(render(f)) == 2


def pease_by_index(x, r, sign=-1):
    """Pease's form in the index terms the kernel uses (z_0 = digit-reversed x;
    stage s: butterfly j takes z[j r + q] * w_{r^s}^(q floor(j / r^(t-s))),
    applies DFT_r and writes z'[p N/r + j]), in complex128."""
    n = x.size
    t = round(math.log(n, r))
    nr = n // r

    def rev(v, m):
        y = 0
        for _ in range(m):
            y, v = y * r + v % r, v // r
        return y

    z = np.array([x[rev(i, t)] for i in range(n)], dtype=np.complex128)
    f = np.exp(sign * 2j * np.pi * np.outer(np.arange(r), np.arange(r)) / r)
    for s in range(1, t + 1):
        zn = np.empty_like(z)
        for j in range(nr):
            k = j // r ** (t - s)
            a = z[j * r + np.arange(r)] * np.exp(sign * 2j * np.pi * np.arange(r) * k / r ** s)
            zn[np.arange(r) * nr + j] = f @ a
        z = zn
    return z


@pytest.mark.parametrize("r,t", [(2, 5), (4, 3), (8, 2), (8, 3), (16, 2), (3, 3), (5, 2)])
def test_pease_index_form_is_the_dft(r, t):
    """Pins the kernel's index form of Pease's stages (both directions) to the oracle's direct DFT."""
    import oracle
    n = r ** t
    x = synth.uniform_batch(synth.DEFAULT_SEED + n, n, 2).astype(np.complex128)
    for sign in (-1, 1):
        ref = oracle.dft_naive(x, sign)
        got = np.stack([pease_by_index(row, r, sign) for row in x])
        assert np.max(np.abs(got - ref)) <= 1e-12 * n, (r, t, sign)


def pease_mutations(r, t):
    """Plausible mistakes in Pease's form (t >= 3): each denotes another matrix."""
    n = r ** t
    good = list(pease(r, t)[1:])
    at = lambda s: 3 * (t - s)  # index of G_s's first factor
    s2 = at(2)
    yield "stage 2 with stage 3's twiddle", good[:s2 + 1] + [kron(tw(r ** 3, r ** 2), eye(r ** (t - 3)))] + good[s2 + 2:]
    yield "twiddle on the other side of its identity", good[:s2 + 1] + [kron(eye(r ** (t - 2)), tw(r ** 2, r))] + good[s2 + 2:]
    yield "stages in reverse order", sum((good[at(s):at(s) + 3] for s in range(1, t + 1)), []) + good[3 * t:]
    yield "digit reversal dropped", good[:3 * t]
    yield "digit reversal applied last", good[3 * t:] + good[:3 * t]
    yield "butterfly factor transposed", [kron(eye(n // r), dft(r))] + good[1:]
    yield "stage permutation Permute(N, N/r)", good[:2] + [perm(n, n // r)] + good[3:]


@pytest.mark.parametrize("r,t", [(2, 3), (3, 3), (4, 3), (2, 4)])
def test_pease_checker_rejects_what_is_not_a_dft(r, t):
    checked = 0
    for why, fs in pease_mutations(r, t):
        f = prod(*fs)
        if not size_ok(f) or is_dft(f):
            continue
        assert checker_accepts(render(f)) is None, why
        assert gbfft.gbfft_formula_form(render(f)) == -1
        checked += 1
    assert checked >= 6


def test_formula_form_codes():
    assert gbfft.gbfft_formula_form("DFT(8)") == 0
    assert gbfft.gbfft_formula_form(render(eq2(dft(4), dft(8)))) == 0
    assert gbfft.gbfft_formula_form(render(eq2_transposed(dft(4), dft(8)))) == 1
    assert gbfft.gbfft_formula_form(render(pease(4, 3))) == 2
    assert gbfft.gbfft_formula_form("I(4)") == -1
    assert gbfft.lib().gbfft_formula_form(None) == -1


# -- formula-driven plans on the GPU -----------------------------------------

def run_formula(text, x, direction=-1):
    import torch
    batch, n = x.shape
    d_in = torch.from_numpy(np.ascontiguousarray(x, np.complex64).view(np.float32).reshape(-1)).cuda()
    d_out = torch.full_like(d_in, float("nan"))
    h, match = gbfft.gbfft_plan_create_formula(text, batch, direction)
    try:
        gbfft.gbfft_execute(h, d_in.data_ptr(), d_out.data_ptr())
        torch.cuda.synchronize()
        info = gbfft.gbfft_plan_info(h)
        k_outer, _ = gbfft.gbfft_plan_factors(h)
    finally:
        gbfft.gbfft_destroy(h)
    return d_out.cpu().numpy().view(np.complex64).reshape(batch, n), match, info, k_outer


@pytest.mark.gpu
def test_eq1_formula_plan_reproduces_the_worked_example():
    import os
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "listing1_dft4.txt"))
    x = (rows[:, 1] + 1j * rows[:, 2]).reshape(1, 4)
    want = rows[:, 3] + 1j * rows[:, 4]
    y, match, info, _ = run_formula(f"var r = {render(eq2(dft(2), dft(2)))} {DOT} Input;", x)
    assert match == 2 and info["radices"] == [2, 2]
    assert np.max(np.abs(y[0] - want)) < 1e-5


@pytest.mark.gpu
@pytest.mark.parametrize("radices,want_match,want_k", [
    ([16, 16, 16], 2, 0),      # a compiled single-pass schedule, same stage order
    ([16, 4, 16], 1, 0),       # the same radices in another order
    ([64, 128], 2, 128),       # N = 8192: Eq. 2 as two passes with the formula's split K = 128
    ([2] * 10, 0, 0),          # no compiled radix-2 schedule: the default plan, still DFT_1024
])
def test_formula_plans_match_the_oracle(radices, want_match, want_k):
    from helpers import ncpu, row_rel_l2, tol_fp32
    import oracle
    n = math.prod(radices)
    x = synth.uniform_batch(synth.DEFAULT_SEED, n, 67)
    y, match, info, k_outer = run_formula(render(ct(radices)), x)
    assert match == want_match
    if want_match == 2 and want_k == 0:
        assert info["radices"] == radices
    if want_k:
        assert k_outer == want_k
    ref = oracle.dft(x.astype(np.complex128), -1, nthreads=ncpu())
    assert row_rel_l2(y, ref).max() <= tol_fp32(n)


@pytest.mark.gpu
@pytest.mark.parametrize("r,t", [(8, 2), (16, 2), (8, 3), (16, 3), (2, 4)])
def test_pease_formula_plans_match_the_oracle(r, t):
    """A Pease formula of a compiled length runs the Pease kernel (variant kind
    5, its radices the formula's leaves); other lengths run the same radices
    as Stockham stages, or the default plan. Both directions against the oracle,
    67 rows (several tiles and a ragged last tile at every length)."""
    from helpers import ncpu, row_rel_l2, tol_fp32
    import oracle
    n = r ** t
    x = synth.uniform_batch(synth.DEFAULT_SEED + n, n, 67)
    for direction in (-1, 1):
        y, match, info, _ = run_formula(render(pease(r, t)), x, direction)
        if n in (64, 256, 512, 4096):
            assert match == 2 and info["radices"] == [r] * t
            assert gbfft.gbfft_variant_kind(n, info["variant"]) == 5
        else:
            assert match in (0, 1)
        ref = oracle.dft(x.astype(np.complex128), direction, nthreads=ncpu())
        assert row_rel_l2(y, ref).max() <= tol_fp32(n), (n, direction)
