"""SVM decision values on the fitted training set (Eq. 1):
f(x) = sum_i alpha_i y_i k(x_i, x) + b, with k the normalised kernel (or K).

The coefficients are given (training the SVM is out of scope); the oracle's
value is its own Khat (or K) times the coefficients in fp64.  The engine
sums n_train products of values within 1e-12 of the oracle's, so the bar is
1e-11 of the sum of absolute terms.  Served values must equal the values of
a single call bit for bit (the reduction order is fixed per row).
"""

import numpy as np
import pytest

import oracle
import paper_1704_07468_gb300 as pkg
from paper_1704_07468_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_07468_gb300 import build as lib_build
    lib_build.build()
    oracle.build()


def _coef(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, n) * (rng.random(n) < 0.4)   # sparse, signed: alpha_i y_i


def _close(f, k, coef, bias):
    ref = k @ coef + bias
    scale = np.abs(k) @ np.abs(coef) + abs(bias)
    assert np.all(np.abs(f - ref) <= 1e-11 * scale + 1e-300), np.max(np.abs(f - ref))


@pytest.mark.parametrize("kind", [0, 1])
def test_decision_values_match_the_oracle(kind):
    tr = synth.random_small(170, 90, 20, 20, 300)
    te = synth.random_small(171, 23, 20, 0, 300)
    coef = _coef(90, 172)
    ref = oracle.cross(te[0], te[1], tr[0], tr[1], 8, 4)
    with pkg.gakco_create(20, 8, 4) as ctx:
        ctx.fit(*tr)
        ctx.set_svm(coef, bias=-0.25, kind=kind)
        f = ctx.decision(*te)
    _close(f, ref["Khat"] if kind == 0 else ref["K"].astype(np.float64), coef, -0.25)


def test_served_decisions_equal_single_calls():
    tr = synth.random_small(173, 70, 4, 40, 250)
    reqs = [synth.random_small(180 + i, int(n), 4, 10, 250) for i, n in enumerate([3, 17, 1, 9, 30, 5])]
    coef = _coef(70, 174)
    with pkg.gakco_create(4, 9, 5) as ctx:
        ctx.set_option("serve_slots", 2)
        ctx.set_option("serve_max_seqs", 20)
        ctx.fit(*tr)
        ctx.set_svm(coef, bias=0.5)
        alone = [ctx.decision(*r) for r in reqs]
        tickets = [ctx.submit(*r, decision=True) for r in reqs]
        served = [ctx.poll(t, timeout_ms=-1) for t in tickets]
    for a, s, r in zip(alone, served, reqs):
        np.testing.assert_array_equal(s["decision"], a)
        ref = oracle.cross(r[0], r[1], tr[0], tr[1], 9, 5)
        _close(a, ref["Khat"], coef, 0.5)


def test_protein_serving_workload_decisions():
    """The serving workload's training set (N = 3312 proteins) and one
    request of its law; sampled rows against the oracle."""
    tr = synth.protein()
    _, c, o = synth.serve_requests(1, seed=9)[0]
    coef = _coef(3312, 175)
    with pkg.gakco_create(20, 8, 4) as ctx:
        ctx.fit(*tr)
        ctx.set_svm(coef, bias=0.1)
        t = ctx.submit(c, o, decision=True, K=False, khat=False)
        out = ctx.poll(t, timeout_ms=-1)
    nt = len(o) - 1
    rows = np.unique(np.array([0, nt - 1, nt // 2], dtype=np.int32))
    ref = oracle.cross(c, o, tr[0], tr[1], 8, 4, rows=rows, threads=len(rows))
    _close(out["decision"][rows], ref["Khat"], coef, 0.1)


def test_svm_errors():
    tr = synth.random_small(176, 12, 4, 20, 80)
    te = synth.random_small(177, 3, 4, 20, 80)
    with pkg.gakco_create(4, 6, 3) as ctx:
        with pytest.raises(pkg.GakcoError):
            ctx.set_svm(np.ones(12))                      # no training set
        ctx.fit(*tr)
        with pytest.raises(pkg.GakcoError):
            ctx.decision(*te)                             # no coefficients
        with pytest.raises(pkg.GakcoError):
            ctx.submit(*te, decision=True)
        with pytest.raises(pkg.GakcoError):
            ctx.set_svm(np.ones(11))                      # wrong length
        with pytest.raises(pkg.GakcoError):
            ctx.set_svm(np.ones(12), kind=2)
        ctx.set_svm(np.ones(12), bias=1.0, kind=1)
        f = ctx.decision(*te)
        ref = oracle.cross(te[0], te[1], tr[0], tr[1], 6, 3)
        _close(f, ref["K"].astype(np.float64), np.ones(12), 1.0)
        ctx.fit(*synth.random_small(178, 12, 4, 20, 80))  # a new training set drops them
        with pytest.raises(pkg.GakcoError):
            ctx.decision(*te)
