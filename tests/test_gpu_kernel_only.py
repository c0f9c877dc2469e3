"""Kernel-only mode: K = C_M.

The coefficients h_m = C(g-m, k) of Eq. 6 equal C(g-m, M-m), the
coefficients of N_m in Eq. 8 at level M, so the kernel is the cumulative
profile of level M alone.  With GAKCO_OPT_KERNEL_ONLY a call that asks for
no N_m computes only the C(g, M) level-M masks; K must equal the oracle's
bit for bit, and Khat the full computation's.
"""

from math import comb

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


CASES = [  # (seed, n, sigma, lo, hi, g, k, dense)
    (140, 60, 4, 50, 250, 10, 6, 0),
    (141, 60, 4, 50, 250, 10, 6, 2),     # level M on the tensor cores
    (142, 45, 20, 20, 300, 8, 4, 0),
    (143, 30, 36, 10, 200, 8, 5, 1),
    (144, 25, 4, 0, 90, 6, 6, 0),        # M = 0: the only level
]


@pytest.mark.parametrize("case", CASES)
def test_kernel_only_matches_the_oracle(case):
    seed, n, sigma, lo, hi, g, k, dense = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    ref = oracle.gram(codes, off, g, k)
    with pkg.gakco_create(sigma, g, k) as ctx:
        ctx.set_option("dense", dense)
        ctx.set_option("kernel_only", 1)
        out = ctx.gram(codes, off, khat=True, nm=False)
        passes = ctx.get_stat("mask_passes")
    np.testing.assert_array_equal(out["K"], ref["K"])
    err = np.abs(out["Khat"] - ref["Khat"])
    assert np.all(err <= KHAT_RTOL * np.abs(ref["Khat"]) + 1e-300)
    assert passes == comb(g, g - k)


def test_kernel_only_equals_the_full_path_in_a_batch():
    sets = [synth.random_small(150 + i, n, 4, 80, 260) for i, n in enumerate([70, 0, 130, 1])]
    with pkg.gakco_create(4, 9, 5) as ctx:
        ctx.set_option("dense", 1)
        full = ctx.gram_batch(sets, khat=True, nm=False)
        ctx.set_option("kernel_only", 1)
        fast = ctx.gram_batch(sets, khat=True, nm=False)
        again = ctx.gram_batch(sets, khat=True, nm=False)
        assert ctx.get_stat("graph_replay") == 1
    for a, b, r in zip(full, fast, again):
        np.testing.assert_array_equal(a["K"], b["K"])
        np.testing.assert_array_equal(a["Khat"], b["Khat"])
        np.testing.assert_array_equal(b["K"], r["K"])


def test_asking_for_the_profile_runs_every_level():
    codes, off = synth.random_small(160, 40, 4, 30, 150)
    ref = oracle.gram(codes, off, 7, 4)
    with pkg.gakco_create(4, 7, 4) as ctx:
        ctx.set_option("kernel_only", 1)
        out = ctx.gram(codes, off, khat=True, nm=True)
        assert ctx.get_stat("mask_passes") == sum(comb(7, m) for m in range(4))
    np.testing.assert_array_equal(out["Nm"], ref["Nm"])
    np.testing.assert_array_equal(out["K"], ref["K"])


def test_plain_engine_ignores_kernel_only():
    codes, off = synth.random_small(161, 20, 4, 30, 100)
    ref = oracle.gram(codes, off, 6, 4)
    with pkg.gakco_create(4, 6, 4) as ctx:
        ctx.set_option("engine", 1)
        ctx.set_option("kernel_only", 1)
        out = ctx.gram(codes, off, khat=True, nm=False)
    np.testing.assert_array_equal(out["K"], ref["K"])
