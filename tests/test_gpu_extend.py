"""Adding sequences to the fitted set (the adaptive training of Section 3.2,
Fig. 5(c)): the Gram matrix of the union from the old Gram matrix, the new
rows' cross kernel and the new block's Gram kernel must equal a fresh Gram
computation on the union, K bit for bit and Khat value for value (same
normalisation formula on both routes), and the oracle on the union.
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
        K0 = ctx.gram(*old, khat=False)["K"]
        ctx.fit(*old)
        ext1 = ctx.extend(*add1, K0)
        ext2 = ctx.extend(*add2, ext1["K"])
        u2 = _union(old, add1, add2)
        fresh = ctx.gram(*u2, khat=True)
        probe = synth.random_small(193, 4, sigma, 30, 200)
        cr = ctx.cross_fitted(*probe)          # the index now holds the union
    np.testing.assert_array_equal(ext2["K"], fresh["K"])
    np.testing.assert_array_equal(ext2["Khat"], fresh["Khat"])
    ref = oracle.gram(*u2, g, k)
    np.testing.assert_array_equal(ext2["K"], ref["K"])
    refx = oracle.cross(probe[0], probe[1], u2[0], u2[1], g, k)
    np.testing.assert_array_equal(cr["K"], refx["K"])


def test_extend_edge_cases():
    old = synth.random_small(194, 8, 4, 20, 80)
    add = synth.random_small(195, 5, 4, 20, 80)
    with pkg.gakco_create(4, 6, 3) as ctx:
        K0 = ctx.gram(*old, khat=False)["K"]
        ctx.fit(*old)
        same = ctx.extend(*synth.pack([]), K0)     # nothing added
        np.testing.assert_array_equal(same["K"], K0)
        ctx.fit(*synth.pack([]))                    # empty fitted set
        ext = ctx.extend(*add, np.zeros((0, 0), np.int32))
        np.testing.assert_array_equal(ext["K"], oracle.gram(*add, 6, 3)["K"])
        ctx.set_svm(np.ones(5))
        ctx.extend(*synth.random_small(196, 2, 4, 20, 80), ext["K"])
        with pytest.raises(pkg.GakcoError):
            ctx.decision(*add)                      # coefficients were dropped
