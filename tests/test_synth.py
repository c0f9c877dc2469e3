"""The seeded stand-ins for the paper's datasets (Table 3; the recipe the
design notes state): sizes, length laws, alphabets and symbol frequencies,
and determinism.  CPU only."""

import numpy as np

from paper_1704_07468_gb300 import synth


def _lengths(off):
    return np.diff(off)


def test_dna_large_recipe():
    sets = synth.dna_large()
    assert [len(o) - 1 for _, o in sets] == [500, 1000, 2000, 3000, 4000]
    allc = np.concatenate([c for c, _ in sets])
    for c, o in sets:
        L = _lengths(o)
        assert L.min() >= 100 and L.max() <= 300
        assert c.max() <= 3
    freq = np.bincount(allc, minlength=4) / allc.size
    np.testing.assert_allclose(freq, [0.3, 0.2, 0.2, 0.3], atol=0.005)  # GC content 0.4
    # independently seeded datasets
    assert not np.array_equal(sets[0][0][:100], sets[1][0][:100])


def test_protein_recipe():
    c, o = synth.protein()
    assert len(o) - 1 == 3312  # SCOP 1.34's size
    L = _lengths(o)
    assert L.min() >= 50 and L.max() <= 1000
    assert 250 <= np.median(L) <= 350  # lognormal around 300
    assert c.max() <= 19


def test_text_recipe():
    c, o = synth.text()
    assert len(o) - 1 == 6000
    L = _lengths(o)
    assert L.min() >= 200 and L.max() <= 2000
    assert c.max() <= 35
    freq = np.bincount(c, minlength=36) / c.size
    # Zipf(1.1) by rank: frequencies fall with the code, f(1) / f(2) = 2^1.1
    assert np.all(np.diff(freq[:10]) < 0)
    np.testing.assert_allclose(freq[0] / freq[1], 2 ** 1.1, rtol=0.02)


def test_serving_requests():
    reqs = synth.serve_requests(400, seed=9)
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) > 0)
    np.testing.assert_allclose(np.mean(np.diff(t)), 0.005, rtol=0.15)  # 200 requests per second
    sizes = np.array([len(o) - 1 for _, _, o in reqs])
    assert sizes.min() >= 1 and sizes.max() <= 256


def test_generators_are_deterministic():
    a, b = synth.protein(seed=7, n=50), synth.protein(seed=7, n=50)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    c, o = synth.pack([np.array([1, 2], np.uint8), np.zeros(0, np.uint8), np.array([3], np.uint8)])
    np.testing.assert_array_equal(o, [0, 2, 2, 3])
    np.testing.assert_array_equal(c, [1, 2, 3])
