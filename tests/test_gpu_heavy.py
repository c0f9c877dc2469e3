"""Heavy features on the tensor cores.

A feature held by L sequences costs about L^2 / 2 pair updates in the
on-chip accumulation (countAndUpdate of Alg. 1), but one column of a dense
contraction.  With GAKCO_OPT_HEAVY (off by default) the batched engine
moves features with
at least T = ceil(heavy * n / 1000) entries (counts all <= 16) of the
sparse levels into e4m3 count matrices and adds A A^T on the tensor cores.
This is an engine choice with no counterpart in the paper, so nothing may
change: K and every N_m bit for bit equal to the oracle's (on sampled rows
at the larger sizes) and to the engine with the option off.
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


def _gram(sigma, g, k, codes, off, **opts):
    with pkg.gakco_create(sigma, g, k) as ctx:
        for name, v in opts.items():
            ctx.set_option(name, v)
        out = ctx.gram(codes, off, khat=True, nm=True)
        out["heavy_columns"] = ctx.get_stat("heavy_columns")
        out["heavy_flops"] = ctx.get_stat("heavy_flops")
    return out


def _same(a, b):
    np.testing.assert_array_equal(a["K"], b["K"])
    np.testing.assert_array_equal(a["Nm"], b["Nm"])
    np.testing.assert_array_equal(a["Khat"], b["Khat"])


def _rows_match_oracle(out, codes, off, g, k, rows):
    ref = oracle.gram(codes, off, g, k, rows=rows)
    np.testing.assert_array_equal(out["K"][rows], ref["K"])
    np.testing.assert_array_equal(out["Nm"][:, rows], ref["Nm"])
    err = np.abs(out["Khat"][rows] - ref["Khat"])
    assert np.all(err <= KHAT_RTOL * np.abs(ref["Khat"]) + 1e-300)


def _sample(n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n - 1, n // 2], rng.integers(0, n, 5)])).astype(np.int32)


def _text_with_repeats(seed, n, lo, hi):
    """Skewed text plus homopolymers whose counts exceed 16 (their features
    must stay on the sparse route)."""
    codes, off = synth.text(seed=seed, n=n, lo=lo, hi=hi)
    seqs = [codes[off[i]:off[i + 1]] for i in range(n)]
    seqs += [np.full(200 + 3 * i, i % 3, dtype=np.uint8) for i in range(6)]
    return synth.pack(seqs)


CASES = [  # (name, sigma, g, k, builder, options)
    ("text", 36, 8, 5, lambda: synth.text(seed=31, n=420, lo=50, hi=400), {"heavy": 20}),
    ("text_repeats", 36, 8, 5, lambda: _text_with_repeats(32, 300, 40, 300), {"heavy": 20}),
    ("dna_dense", 4, 10, 6, lambda: synth.dna_large(seeds=(33,), sizes=(300,))[0], {"dense": 1, "heavy": 5}),
    ("dna_low_T", 4, 8, 4, lambda: synth.random_small(34, 280, 4, 60, 260), {"heavy": 1}),
    ("protein", 20, 8, 4, lambda: synth.protein(seed=35, n=300), {"heavy": 5}),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_heavy_features_change_nothing(case):
    name, sigma, g, k, build, opts = case
    codes, off = build()
    n = len(off) - 1
    on = _gram(sigma, g, k, codes, off, **opts)
    off_ = _gram(sigma, g, k, codes, off, **{**opts, "heavy": 0})
    assert on["heavy_columns"] > 0, "no feature took the dense route"
    assert off_["heavy_columns"] == 0
    _same(on, off_)
    _rows_match_oracle(on, codes, off, g, k, _sample(n, 7))


def test_column_budget_leaves_the_rest_sparse():
    codes, off = synth.text(seed=36, n=300, lo=50, hi=300)
    full = _gram(36, 8, 5, codes, off, heavy=20)
    # Level 3 (56 of the 93 masks) gets 60 % of the budget: one block of 128
    # columns of 384 rows; the other levels' shares fall below one block.
    tight = _gram(36, 8, 5, codes, off, heavy=20, heavy_bytes=100000)
    none = _gram(36, 8, 5, codes, off, heavy=20, heavy_bytes=0)
    assert 0 < tight["heavy_columns"] < full["heavy_columns"]
    assert none["heavy_columns"] == 0
    _same(full, tight)
    _same(full, none)


def test_threshold_extremes_and_small_sets():
    codes, off = synth.text(seed=37, n=260, lo=30, hi=200)
    ref = _gram(36, 8, 5, codes, off, heavy=0)
    all_heavy = _gram(36, 8, 5, codes, off, heavy=1)       # T = 8 entries
    no_heavy = _gram(36, 8, 5, codes, off, heavy=1000)     # T = n: a feature in every sequence
    _same(ref, all_heavy)
    _same(ref, no_heavy)
    small = synth.text(seed=38, n=200, lo=30, hi=200)      # below 256 sequences: all sparse
    out = _gram(36, 8, 5, *small, heavy=20)
    assert out["heavy_columns"] == 0
    _same(out, _gram(36, 8, 5, *small, heavy=0))


def test_replay_batch_and_kernel_only():
    sets = [synth.text(seed=40 + i, n=n, lo=40, hi=300) for i, n in enumerate([300, 0, 280, 5])]
    with pkg.gakco_create(36, 8, 5) as ctx:
        ctx.set_option("heavy", 20)
        a = ctx.gram_batch(sets, khat=True, nm=True)
        cols = ctx.get_stat("heavy_columns")
        b = ctx.gram_batch(sets, khat=True, nm=True)
        assert ctx.get_stat("graph_replay") == 1
        assert ctx.get_stat("heavy_columns") == cols > 0
        ctx.set_option("kernel_only", 1)
        c = ctx.gram_batch(sets, khat=True, nm=False)
        ctx.set_option("heavy", 0)
        d = ctx.gram_batch(sets, khat=True, nm=True)
    for x, y, z, r in zip(a, b, c, d):
        _same(x, y)
        _same(x, r)
        np.testing.assert_array_equal(z["K"], r["K"])
        np.testing.assert_array_equal(z["Khat"], r["Khat"])
    codes, off = sets[0]
    ref = oracle.gram(codes, off, 8, 5, rows=_sample(300, 8))
    np.testing.assert_array_equal(a[0]["K"][_sample(300, 8)], ref["K"])
