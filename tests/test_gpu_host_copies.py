"""Host-buffer outputs: the same values whichever way they reach the
caller (GAKCO_OPT_DIRECT_D2H: pinned staging, direct copies into the
caller's first-touched pages, or the automatic choice), for outputs above
the 8 MiB size from which both paths differ, for a batched Gram call and a
cross kernel, and equal to the device-buffer call."""

import numpy as np
import pytest
import torch

import paper_1704_07468_gb300 as pkg
from paper_1704_07468_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_07468_gb300 import build as lib_build
    lib_build.build()


def test_copy_modes_agree():
    sets = [synth.random_small(210, 1100, 4, 40, 200), synth.random_small(211, 700, 4, 40, 200)]
    test = synth.random_small(212, 900, 4, 40, 200)
    outs, crosses = [], []
    for mode in (0, 1, -1):
        with pkg.gakco_create(4, 8, 5) as ctx:
            ctx.set_option("direct_d2h", mode)
            outs.append(ctx.gram_batch(sets, khat=True, nm=True))
            ctx.fit(*sets[0])
            crosses.append(ctx.cross_fitted(*test))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            for key in ("K", "Khat", "Nm"):
                np.testing.assert_array_equal(a[key], b[key])
    for x in crosses[1:]:
        np.testing.assert_array_equal(crosses[0]["K"], x["K"])
        np.testing.assert_array_equal(crosses[0]["Khat"], x["Khat"])
    # and the device-buffer call
    dev = torch.device("cuda:0")
    codes, off = sets[0]
    n = len(off) - 1
    d_codes = torch.from_numpy(codes).to(dev)
    d_K = torch.empty((n, n), dtype=torch.int32, device=dev)
    with pkg.gakco_create(4, 8, 5) as ctx:
        ctx.gram_batch_device([d_codes.data_ptr()], [off], [d_K.data_ptr()], None, None)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(d_K.cpu().numpy(), outs[0][0]["K"])


def test_copy_mode_validation():
    with pkg.gakco_create(4, 6, 3) as ctx:
        for bad in (-2, 2):
            with pytest.raises(pkg.GakcoError):
                ctx.set_option("direct_d2h", bad)
