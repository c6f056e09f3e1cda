"""The seeded input generator: deterministic, counter-based, exact in float32,
and identical whether a batch is drawn whole or row by row."""
import numpy as np

from paper_2207_06803_gb300 import synth

MASK = (1 << 64) - 1


def splitmix64_scalar(seed, count):
    """SplitMix64 as published (Steele, Lea, Flood 2014), one word at a time."""
    state, out = seed & MASK, []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


def test_words_match_sequential_splitmix64():
    for seed in (0, 1, 20220714, MASK):
        assert synth.words(seed, 0, 64).tolist() == splitmix64_scalar(seed, 64)
        assert synth.words(seed, 17, 5).tolist() == splitmix64_scalar(seed, 22)[17:]


def test_uniform_range_lattice_and_determinism():
    a = synth.uniform_flat(7, 0, 1 << 16)
    f = a.view(np.float32)
    assert f.min() >= -1.0 and f.max() < 1.0
    # every value is k * 2^-23 - 1 for an integer k < 2^24: exact in float32
    k = (f.astype(np.float64) + 1.0) * 2.0 ** 23
    assert np.array_equal(k, np.round(k))
    assert np.array_equal(a, synth.uniform_flat(7, 0, 1 << 16))
    assert not np.array_equal(a, synth.uniform_flat(8, 0, 1 << 16))
    assert abs(float(f.mean())) < 0.01


def test_rows_equal_slices_of_batch():
    b = synth.uniform_batch(3, 48, 20)
    assert np.array_equal(synth.uniform_rows(3, 48, [0, 5, 19]), b[[0, 5, 19]])
    g = synth.gaussian_scaled_batch(3, 40, 12)
    assert np.array_equal(synth.gaussian_scaled_rows(3, 40, [0, 7, 11]), g[[0, 7, 11]])


def test_gaussian_rows_scaled_between_1e_minus_3_and_1e3():
    g = synth.gaussian_scaled_batch(11, 256, 400).astype(np.complex128)
    rms = np.sqrt(np.mean(np.abs(g) ** 2, axis=1) / 2)
    assert rms.min() > 1e-3 / 2 and rms.max() < 1e3 * 2
    assert np.log10(rms).std() > 1.2  # spread over about six decades


def test_size_family_has_41_sizes_in_8_8192():
    fam = synth.size_family(8, 8192)
    assert len(fam) == 41 and fam[0] == 8 and fam[-1] == 8192
    for n in fam:
        m = n
        while m % 2 == 0:
            m //= 2
        assert m in (1, 3, 5, 7)
    sizes = synth.ragged_sizes(1, 10000)
    assert set(sizes.tolist()) <= set(fam) and len(set(sizes.tolist())) == 41
    off = synth.ragged_offsets(sizes)
    assert off[0] == 0 and np.all(np.diff(off) == sizes[:-1])


def test_sample_rows_distinct_sorted():
    r = synth.sample_rows(5, 1000, 100)
    assert len(set(r.tolist())) == 100 and np.all(np.diff(r) > 0) and r.max() < 1000
