"""Adding sequences to the fitted set (the adaptive training of Section 3.2,
Fig. 5(c)): the new rows of the union's Gram matrix, from the resident
index (cross kernel) and the new block's Gram kernel, must equal the rows
of a fresh Gram computation on the union, K bit for bit and Khat value for
value (same normalisation formula and operand order), and the oracle.  The
resident index is then the new sequences' index merged into the old one; it
must answer exactly like an index fitted on the union.
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


def _union(*sets):
    seqs = []
    for c, o in sets:
        seqs += [c[o[i]:o[i + 1]] for i in range(len(o) - 1)]
    return synth.pack(seqs)


@pytest.mark.parametrize("sigma,g,k", [(4, 10, 6), (20, 8, 4)])
def test_extend_equals_a_fresh_gram(sigma, g, k):
    old = synth.random_small(190, 50, sigma, 30, 260)
    add1 = synth.random_small(191, 17, sigma, 0, 260)
    add2 = synth.random_small(192, 6, sigma, 30, 260)
    with pkg.gakco_create(sigma, g, k) as ctx:
        ctx.set_option("dense", 1)
        ctx.fit(*old)
        rows1 = ctx.extend(*add1)
        rows2 = ctx.extend(*add2)
        u1, u2 = _union(old, add1), _union(old, add1, add2)
        fresh1 = ctx.gram(*u1, khat=True)
        fresh2 = ctx.gram(*u2, khat=True)
        probe = synth.random_small(193, 4, sigma, 30, 200)
        cr = ctx.cross_fitted(*probe)          # the index now holds the union
    np.testing.assert_array_equal(rows1["K"], fresh1["K"][50:])
    np.testing.assert_array_equal(rows1["Khat"], fresh1["Khat"][50:])
    np.testing.assert_array_equal(rows2["K"], fresh2["K"][67:])
    np.testing.assert_array_equal(rows2["Khat"], fresh2["Khat"][67:])
    ref = oracle.gram(*u2, g, k, rows=np.arange(67, 73, dtype=np.int32))
    np.testing.assert_array_equal(rows2["K"], ref["K"])
    refx = oracle.cross(probe[0], probe[1], u2[0], u2[1], g, k)
    np.testing.assert_array_equal(cr["K"], refx["K"])


def test_extend_edge_cases():
    old = synth.random_small(194, 8, 4, 20, 80)
    add = synth.random_small(195, 5, 4, 20, 80)
    with pkg.gakco_create(4, 6, 3) as ctx:
        ctx.fit(*old)
        none = ctx.extend(*synth.pack([]))          # nothing added
        assert none["K"].shape == (0, 8)
        ctx.fit(*synth.pack([]))                    # empty fitted set
        rows = ctx.extend(*add)
        np.testing.assert_array_equal(rows["K"], oracle.gram(*add, 6, 3)["K"])
        ctx.set_svm(np.ones(5))
        ctx.extend(*synth.random_small(196, 2, 4, 20, 80))
        with pytest.raises(pkg.GakcoError):
            ctx.decision(*add)                      # coefficients were dropped


@pytest.mark.parametrize("sigma,g,k", [(4, 10, 6), (20, 8, 4), (36, 8, 5)])
def test_merged_index_equals_a_fit_of_the_union(sigma, g, k):
    """Several extends in a row (one sequence, empty and short sequences,
    a larger block): the merged index must answer exactly like an index
    fitted on the union (cross kernels and decision values bit for bit)."""
    old = synth.random_small(200, 40, sigma, 30, 220)
    adds = [synth.random_small(201, 1, sigma, 30, 200),
            synth.random_small(202, 7, sigma, 0, 12),        # empty and shorter-than-g sequences
            synth.random_small(203, 33, sigma, 30, 260)]
    probe = synth.random_small(204, 9, sigma, 0, 240)
    u = _union(old, *adds)
    nu = len(u[1]) - 1
    coef = np.random.default_rng(205).uniform(-1, 1, nu)
    with pkg.gakco_create(sigma, g, k) as ctx:
        ctx.fit(*old)
        for a in adds:
            ctx.extend(*a)
        merged = ctx.cross_fitted(*probe)
        ctx.set_svm(coef, bias=0.3)
        f_merged = ctx.decision(*probe)
    with pkg.gakco_create(sigma, g, k) as ctx:
        ctx.fit(*u)
        fresh = ctx.cross_fitted(*probe)
        ctx.set_svm(coef, bias=0.3)
        f_fresh = ctx.decision(*probe)
    np.testing.assert_array_equal(merged["K"], fresh["K"])
    np.testing.assert_array_equal(merged["Khat"], fresh["Khat"])
    np.testing.assert_array_equal(f_merged, f_fresh)
    ref = oracle.cross(probe[0], probe[1], u[0], u[1], g, k)
    np.testing.assert_array_equal(merged["K"], ref["K"])


def test_extend_at_the_dna_benchmark_size():
    """The bench's extend case: 100 sequences added to 3900 of the N = 4000
    DNA dataset; the rows against a fresh Gram of all 4000 on sampled rows,
    and cross kernels of the merged index against a fitted one."""
    codes, off = synth.dna_large(sizes=(4000,), seeds=(6,))[0]
    seqs = [codes[off[i]:off[i + 1]] for i in range(4000)]
    old, new = synth.pack(seqs[:3900]), synth.pack(seqs[3900:])
    probe = synth.random_small(206, 5, 4, 100, 300)
    with pkg.gakco_create(4, 10, 6) as ctx:
        ctx.set_option("dense", 1)
        ctx.fit(*old)
        rows = ctx.extend(*new)
        merged = ctx.cross_fitted(*probe)
        full = ctx.gram(codes, off, khat=True)
        ctx.fit(codes, off)
        fresh = ctx.cross_fitted(*probe)
    np.testing.assert_array_equal(rows["K"], full["K"][3900:])
    np.testing.assert_array_equal(rows["Khat"], full["Khat"][3900:])
    np.testing.assert_array_equal(merged["K"], fresh["K"])
    np.testing.assert_array_equal(merged["Khat"], fresh["Khat"])
    sample = np.array([0, 57, 99], dtype=np.int32)
    ref = oracle.gram(codes, off, 10, 6, rows=sample + 3900, threads=len(sample))
    np.testing.assert_array_equal(rows["K"][sample], ref["K"])
