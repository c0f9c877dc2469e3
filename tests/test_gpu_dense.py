"""Dense levels on the tensor cores: C_m += A A^T with A the per-sequence
counts of every (mask, (g-m)-mer) of a level (countAndUpdate of Alg. 1 as a
dense contraction).

The route is exact integer arithmetic (counts up to 16 in e4m3, f32 partial
sums flushed to int32 before 2^24, larger counts corrected from an overflow
list), so every integer output must equal the oracle's bit for bit, and
equal the sparse route's.
"""

import numpy as np
import pytest

import oracle
import paper_1704_07468_gb300 as pkg
from paper_1704_07468_gb300 import synth

pytestmark = pytest.mark.gpu
KHAT_RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_07468_gb300 import build as lib_build
    lib_build.build()
    oracle.build()


def _run(sigma, g, k, codes, off, **opts):
    with pkg.gakco_create(sigma, g, k) as ctx:
        for name, v in opts.items():
            ctx.set_option(name, v)
        out = ctx.gram(codes, off, khat=True, nm=True)
        out["dense_problems"] = ctx.get_stat("dense_problems")
        out["dense_flops"] = ctx.get_stat("dense_flops")
    return out


def _check(out, ref):
    np.testing.assert_array_equal(out["K"], ref["K"])
    np.testing.assert_array_equal(out["Nm"], ref["Nm"])
    err = np.abs(out["Khat"] - ref["Khat"])
    assert np.all(err <= KHAT_RTOL * np.abs(ref["Khat"]) + 1e-300)


CASES = [  # (seed, n, sigma, lo, hi, g, k)
    (120, 40, 4, 100, 300, 10, 6),    # DNA large-M shape: level 4 (4096 keys) dense
    (121, 260, 4, 0, 200, 8, 4),      # three row blocks, ragged n, partial B tile
    (122, 30, 4, 10, 120, 10, 3),     # M = 7: levels 5..7 have 10, 8, 6 key bits
    (123, 25, 2, 0, 80, 4, 1),        # binary alphabet: 2..16-column masks, rows padded to 128 columns
    (124, 19, 3, 5, 60, 6, 2),        # sigma = 3 (2 bits per symbol, code 3 unused)
    (125, 9, 4, 10, 40, 5, 5),        # M = 0: the spectrum level alone
    (126, 30, 4, 20, 150, 13, 7),     # 26-bit full keys: four byte tables per mask
]


@pytest.mark.parametrize("case", CASES)
def test_dense_levels_match_the_oracle(case):
    seed, n, sigma, lo, hi, g, k = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    ref = oracle.gram(codes, off, g, k)
    out = _run(sigma, g, k, codes, off, dense=2)
    assert out["dense_problems"] > 0
    _check(out, ref)


@pytest.mark.parametrize("case", CASES[:3])
def test_dense_gemm_after_the_sparse_passes_is_exact(case):
    seed, n, sigma, lo, hi, g, k = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    ref = oracle.gram(codes, off, g, k)
    out = _run(sigma, g, k, codes, off, dense=2, dense_late=1)
    assert out["dense_problems"] > 0
    _check(out, ref)


@pytest.mark.parametrize("case", CASES[:3])
def test_dense_tail_split_is_exact(case):
    """K-parts of the last wave's tiles (and of every tile when there are
    fewer tiles than CTAs) change nothing."""
    seed, n, sigma, lo, hi, g, k = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    ref = oracle.gram(codes, off, g, k)
    for sms in (0, 3):
        out = _run(sigma, g, k, codes, off, dense=2, dense_split=1, dense_sms=sms)
        assert out["dense_problems"] > 0
        _check(out, ref)
        # Kernel-only mode with a dense top level: no sparse level at all,
        # so the automatic choice splits.
        with pkg.gakco_create(sigma, g, k) as ctx:
            for name, v in (("dense", 2), ("dense_split", -1), ("kernel_only", 1), ("dense_sms", sms)):
                ctx.set_option(name, v)
            ko = ctx.gram(codes, off, khat=True, nm=False)
            assert ctx.get_stat("dense_problems") > 0
        np.testing.assert_array_equal(ko["K"], ref["K"])
        assert np.all(np.abs(ko["Khat"] - ref["Khat"]) <= KHAT_RTOL * np.abs(ref["Khat"]) + 1e-300)


def test_dense_equals_sparse_on_several_waves():
    """A small wave budget cuts each level into several mask runs and the
    runs into several waves; the result must not change."""
    codes, off = synth.random_small(126, 300, 4, 100, 300)
    g, k = 9, 5
    sparse = _run(4, g, k, codes, off, dense=0)
    assert sparse["dense_problems"] == 0
    n_pad = 384
    one_mask = n_pad * 4 ** 5                # level 4: 5-mers, one byte each
    dense = _run(4, g, k, codes, off, dense=2, dense_bytes=3 * one_mask)
    assert dense["dense_problems"] > 10
    for key in ("K", "Nm", "Khat"):
        np.testing.assert_array_equal(dense[key], sparse[key])
    rows = np.array([0, 127, 128, 255, 299], dtype=np.int32)
    ref = oracle.gram(codes, off, g, k, rows=rows)
    np.testing.assert_array_equal(dense["K"][rows], ref["K"])


@pytest.mark.parametrize("kind", ["homopolymer", "period2", "mixed"])
def test_large_counts_are_corrected_exactly(kind):
    """Counts of 496 for one feature per mask: A holds 16 and the overflow
    list carries the rest."""
    codes, off = synth.repeats(kind, n=4, length=500)
    ref = oracle.gram(codes, off, 5, 3)
    out = _run(4, 5, 3, codes, off, dense=2)
    assert out["dense_problems"] > 0
    _check(out, ref)


def test_overflows_sharing_a_column():
    """Homopolymers of one symbol: every sequence overflows at the same
    column of every mask, so the pair terms of the correction meet; lengths
    around g + 15 put counts at 15, 16, 17 and 18 (the e4m3 edge)."""
    g, k = 6, 3
    lens = [g + 14, g + 15, g + 16, g + 17, 40, 100, 7, 0, 300]
    seqs = [np.zeros(n, np.uint8) for n in lens]
    seqs += [np.full(60, 2, np.uint8), np.array([0, 1] * 40, np.uint8)]
    codes, off = synth.pack(seqs)
    ref = oracle.gram(codes, off, g, k)
    out = _run(4, g, k, codes, off, dense=2)
    assert out["dense_problems"] > 0
    _check(out, ref)


def test_every_count_value_is_encoded_exactly():
    """A homopolymer of length g - 1 + c holds one column of count c in
    every mask, for c = 0..20: each count 1..7 goes through the scatter's
    table of e4m3 bytes, 8..16 through the f16 conversion, 17..20 through
    the overflow list.  Mixed with random rows and two-symbol blocks, whose
    counts share 8-column words with other counts."""
    g, k = 6, 3
    rng = np.random.default_rng(130)
    seqs = [np.full(g - 1 + c, c % 4, np.uint8) for c in range(21)]
    seqs += [np.concatenate([np.zeros(g - 1 + a, np.uint8), np.ones(g - 1 + b, np.uint8)])
             for a, b in ((3, 9), (7, 8), (12, 2), (16, 17))]
    seqs += [rng.integers(0, 4, int(n), dtype=np.uint8) for n in rng.integers(5, 90, 12)]
    codes, off = synth.pack(seqs)
    ref = oracle.gram(codes, off, g, k)
    out = _run(4, g, k, codes, off, dense=2)
    assert out["dense_problems"] > 0
    _check(out, ref)


def test_full_overflow_list_reruns_sparse():
    """An overflow list too small for the input: the call reruns with every
    level sparse and stays exact."""
    codes, off = synth.repeats("mixed", n=6, length=400)
    ref = oracle.gram(codes, off, 5, 2)
    out = _run(4, 5, 2, codes, off, dense=2, dense_overflow=2)
    assert out["dense_problems"] == 0     # the rerun planned every level sparse
    _check(out, ref)


def test_long_sequences_go_dense():
    """More than 511 windows per sequence: counts are not bounded by the
    e4m3 range, which the overflow list covers."""
    codes, off = synth.random_small(127, 6, 4, 500, 700)
    ref = oracle.gram(codes, off, 6, 3)
    out = _run(4, 6, 3, codes, off, dense=2)
    assert out["dense_problems"] > 0
    _check(out, ref)


def test_dense_batch_and_graph_replay():
    sets = [synth.random_small(130 + i, n, 4, 80, 250) for i, n in enumerate([50, 1, 0, 140])]
    with pkg.gakco_create(4, 8, 5) as ctx:
        ctx.set_option("dense", 2)
        first = ctx.gram_batch(sets, khat=True, nm=True)
        probs = ctx.get_stat("dense_problems")
        again = ctx.gram_batch(sets, khat=True, nm=True)
        assert ctx.get_stat("graph_replay") == 1
        assert ctx.get_stat("dense_problems") == probs > 0
    for (c, o), a, b in zip(sets, first, again):
        for key in ("K", "Nm", "Khat"):
            np.testing.assert_array_equal(a[key], b[key])
        if len(o) > 1:
            _check(a, oracle.gram(c, o, 8, 5))


def test_cost_model_mode_is_exact():
    codes, off = synth.random_small(128, 200, 4, 100, 300)
    out = _run(4, 10, 6, codes, off, dense=1)
    sparse = _run(4, 10, 6, codes, off, dense=0)
    for key in ("K", "Nm", "Khat"):
        np.testing.assert_array_equal(out[key], sparse[key])


def test_dna_large_dataset_sampled_rows():
    """The N = 4000 dataset of the DNA large-M workload (g = 10, k = 6) with
    every qualifying level dense; sampled rows against the oracle."""
    codes, off = synth.dna_large(seeds=[6], sizes=[4000])[0]
    out = _run(4, 10, 6, codes, off, dense=2)
    assert out["dense_problems"] > 0
    rows = np.array([0, 1, 1999, 3998, 3999], dtype=np.int32)
    ref = oracle.gram(codes, off, 10, 6, rows=rows, threads=len(rows))
    np.testing.assert_array_equal(out["K"][rows], ref["K"])
    np.testing.assert_array_equal(out["Nm"][:, rows], ref["Nm"])
    np.testing.assert_array_equal(out["K"], out["K"].T)
