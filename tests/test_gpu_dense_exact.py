"""The dense GEMM's exact accumulation rounds, its multi-round path and its
bounded waits.

Dense levels add A A^T (A: per-sequence counts min(c, 16) of every
(mask, (g-m)-mer), in e4m3) on the tensor cores with f32 accumulators in
tensor memory, and move a round into the int32 C_m before any partial sum
can pass 2^24 - 1 (countAndUpdate of Alg. 1, summed as in Eq. 8).  A round
covers a whole macro tile when a row's largest possible sum, 16 x windows
x masks, stays within that bound.

* Periodic sequences in which every masked key recurs 16 times push the
  real partial sums of one round to just below 2^24 (about 2^23.99), so
  the tensor cores' integer accumulation is checked against the oracle over
  the whole range the engine relies on.
* A lowered round bound runs the same inputs, ordinary ones and the
  heavy-feature GEMM through many rounds (the atomic epilogue).
* A role-wait limit of a few cycles makes the GEMM's waits run out: the
  call returns GAKCO_E_TIMEOUT, and the context then computes correctly.
"""

from itertools import combinations

import numpy as np
import pytest

import oracle
import paper_1704_07468_gb300 as pkg
from paper_1704_07468_gb300 import synth

pytestmark = pytest.mark.gpu
KHAT_RTOL = 1e-12
EXACT = (1 << 24) - 1

# g = 12, k = 7: levels 4 (8-mers, 495 masks) and 5 (7-mers, 792 masks)
# have keys of at most 16 bits and go dense.  With 1312 windows (period 82,
# 16 copies) a level-5 row sums to 16 x 1312 x 792 = 16,625,664 <= 2^24 - 1
# at most, so the engine takes one round per macro tile; the int32 bound
# 792 x 1312^2 < 2^31 holds.
G, K = 12, 7
PERIOD = 82


def _periodic_set():
    codes, off = synth.periodic(seed=140, period=PERIOD,
                                lengths=[16 * PERIOD + G - 1, 16 * PERIOD + G - 1,
                                         8 * PERIOD + G - 1, 400],
                                shifts=[0, 40, 17, 3])
    rnd, roff = synth.random_small(141, 3, 4, 5, 300)
    seqs = [codes[off[i]:off[i + 1]] for i in range(len(off) - 1)]
    seqs += [rnd[roff[i]:roff[i + 1]] for i in range(len(roff) - 1)]
    return synth.pack(seqs)


def _row_square_sum(seq, g, m, sigma=4, cap=16):
    """sum over the level's masks and keys of min(count, cap)^2 for one
    sequence: the diagonal entry of A A^T, i.e. the final partial sum of its
    accumulator when the level is one round."""
    win = np.lib.stride_tricks.sliding_window_view(seq.astype(np.int64), g)
    total = 0
    for deleted in combinations(range(g), m):
        key = np.zeros(len(win), dtype=np.int64)
        for p in range(g):
            if p not in deleted:
                key = key * sigma + win[:, p]
        _, cnt = np.unique(key, return_counts=True)
        total += int(np.sum(np.minimum(cnt, cap) ** 2))
    return total


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_07468_gb300 import build as lib_build
    lib_build.build()
    oracle.build()


@pytest.fixture(scope="module")
def periodic():
    codes, off = _periodic_set()
    return codes, off, oracle.gram(codes, off, G, K)


def _gram(sigma, g, k, codes, off, **opts):
    with pkg.gakco_create(sigma, g, k) as ctx:
        for name, v in opts.items():
            ctx.set_option(name, v)
        out = ctx.gram(codes, off, khat=True, nm=True)
        out["dense_problems"] = ctx.get_stat("dense_problems")
    return out


def _check(out, ref):
    np.testing.assert_array_equal(out["K"], ref["K"])
    np.testing.assert_array_equal(out["Nm"], ref["Nm"])
    err = np.abs(out["Khat"] - ref["Khat"])
    assert np.all(err <= KHAT_RTOL * np.abs(ref["Khat"]) + 1e-300)


def test_periodic_input_reaches_the_top_of_the_f32_range(periodic):
    """Precondition of the next test, from the inputs alone: the level-5
    accumulators of the periodic sequences end within 1 % of 2^24, and the
    engine's one-round rule applies (16 x windows x masks <= 2^24 - 1)."""
    codes, off, _ = periodic
    seq = codes[off[0]:off[1]]
    w = len(seq) - G + 1
    assert 16 * w * 792 <= EXACT
    top = _row_square_sum(seq, G, 5)
    assert 0.99 * 2 ** 24 < top <= EXACT, top
    assert _row_square_sum(seq, G, 4) > 2 ** 23


def test_one_round_partial_sums_near_2_24_are_exact(periodic):
    codes, off, ref = periodic
    out = _gram(4, G, K, codes, off, dense=2)
    assert out["dense_problems"] > 0
    _check(out, ref)


def test_sparse_route_agrees_on_the_periodic_input(periodic):
    codes, off, ref = periodic
    out = _gram(4, G, K, codes, off, dense=0)
    assert out["dense_problems"] == 0
    _check(out, ref)


@pytest.mark.parametrize("cap", [(1 << 20) - 1, (1 << 22) - 1])
def test_multi_round_path_on_the_periodic_input(periodic, cap):
    codes, off, ref = periodic
    out = _gram(4, G, K, codes, off, dense=2, dense_round_sum=cap)
    _check(out, ref)


@pytest.mark.parametrize("case", [  # (seed, n, lo, hi, g, k, cap)
    (142, 40, 100, 300, 10, 6, 1),            # one stage per round
    (143, 300, 0, 200, 8, 4, 5000),           # several row blocks, a few stages per round
    (144, 30, 1000, 1500, 10, 6, 1 << 21),
])
def test_multi_round_path_matches_the_oracle(case):
    seed, n, lo, hi, g, k, cap = case
    codes, off = synth.random_small(seed, n, 4, lo, hi)
    ref = oracle.gram(codes, off, g, k)
    out = _gram(4, g, k, codes, off, dense=2, dense_round_sum=cap)
    assert out["dense_problems"] > 0
    _check(out, ref)


def test_heavy_feature_gemm_in_single_stage_rounds():
    """The heavy-feature GEMM has no one-round bound and always counts
    rounds by stages; one stage per round must change nothing."""
    codes, off = synth.text(seed=145, n=420, lo=50, hi=400)
    on = _gram(36, 8, 5, codes, off, heavy=20, dense_round_sum=1)
    off_ = _gram(36, 8, 5, codes, off, heavy=0)
    for key in ("K", "Nm", "Khat"):
        np.testing.assert_array_equal(on[key], off_[key])
    rows = np.array([0, 17, 209, 419], dtype=np.int32)
    ref = oracle.gram(codes, off, 8, 5, rows=rows)
    np.testing.assert_array_equal(on["K"][rows], ref["K"])
    np.testing.assert_array_equal(on["Nm"][:, rows], ref["Nm"])


def test_round_bound_option_limits():
    with pkg.gakco_create(4, 10, 6) as ctx:
        for bad in (0, -1, EXACT + 1):
            with pytest.raises(pkg.GakcoError):
                ctx.set_option("dense_round_sum", bad)
        ctx.set_option("dense_round_sum", EXACT)
        with pytest.raises(pkg.GakcoError):
            ctx.set_option("dense_wait_cycles", -1)


def test_gemm_wait_timeout_leaves_the_context_usable():
    """With a role-wait limit of one cycle the epilogue's first wait for a
    finished round runs out (a round needs its copies and MMAs first): every
    role stops, the copies and MMAs already issued are drained, tensor
    memory is freed, and the call reports GAKCO_E_TIMEOUT.  The same context
    then computes the Gram matrix correctly with the default limit."""
    codes, off = synth.random_small(146, 40, 4, 100, 300)
    ref = oracle.gram(codes, off, 10, 6)
    with pkg.gakco_create(4, 10, 6) as ctx:
        ctx.set_option("dense", 2)
        ctx.set_option("dense_wait_cycles", 1)
        with pytest.raises(pkg.GakcoError) as exc:
            ctx.gram(codes, off, khat=True, nm=True)
        assert exc.value.name == "GAKCO_E_TIMEOUT"
        assert "wait" in ctx.last_error()
        ctx.set_option("dense_wait_cycles", 0)
        out = ctx.gram(codes, off, khat=True, nm=True)
        assert ctx.get_stat("dense_problems") > 0
    _check(out, ref)
