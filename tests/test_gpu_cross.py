"""Cross kernel K(test, train) and the serving loop, against the oracle.

The paper classifies with one kernel over training and test sequences
together (Section 3.1); the cross kernel is its test-rows x train-columns
block, with each test diagonal from the test sequence alone.  Integer K is
bit-exact with the oracle; Khat within 1e-12 relative.  Served requests must
give the same rows whether they ran alone or batched with others.
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


def _close(a, b):
    return np.all(np.abs(a - b) <= KHAT_RTOL * np.abs(b) + 1e-300)


CASES = [  # (seed, sigma, g, k, ntrain, ntest, lo, hi)
    (80, 4, 6, 3, 40, 17, 0, 200),
    (81, 20, 8, 4, 55, 9, 30, 300),
    (82, 36, 8, 5, 30, 12, 5, 250),
    (83, 4, 10, 6, 25, 25, 8, 150),
    (84, 3, 5, 5, 20, 7, 0, 60),
]


@pytest.mark.parametrize("case", CASES)
def test_cross_matches_oracle(case):
    seed, sigma, g, k, ntr, nte, lo, hi = case
    tr = synth.random_small(seed, ntr, sigma, lo, hi)
    te = synth.random_small(seed + 100, nte, sigma, lo, hi)
    ref = oracle.cross(te[0], te[1], tr[0], tr[1], g, k)
    with pkg.gakco_create(sigma, g, k) as ctx:
        out = ctx.cross(te, tr)
    np.testing.assert_array_equal(out["K"], ref["K"])
    assert _close(out["Khat"], ref["Khat"])


def test_cross_is_the_block_of_the_joint_gram_on_the_gpu():
    tr = synth.random_small(90, 60, 20, 20, 300)
    te = synth.random_small(91, 20, 20, 20, 300)
    both_c = np.concatenate([tr[0], te[0]])
    both_o = np.concatenate([tr[1], te[1][1:] + tr[1][-1]])
    with pkg.gakco_create(20, 8, 4) as ctx:
        joint = ctx.gram(both_c, both_o, khat=True)
        cr = ctx.cross(te, tr)
    np.testing.assert_array_equal(cr["K"], joint["K"][60:, :60])
    assert _close(cr["Khat"], joint["Khat"][60:, :60])


@pytest.mark.parametrize("cols", [1, 13, 64])
def test_cross_column_tiles(cols):
    tr = synth.random_small(92, 70, 4, 10, 150)
    te = synth.random_small(93, 11, 4, 10, 150)
    ref = oracle.cross(te[0], te[1], tr[0], tr[1], 7, 4)
    with pkg.gakco_create(4, 7, 4) as ctx:
        ctx.set_option("smem_cols", cols)
        out = ctx.cross(te, tr)
    np.testing.assert_array_equal(out["K"], ref["K"])


def test_cross_with_repetitive_sequences():
    tr = synth.repeats("mixed", n=6, length=500)
    te = synth.repeats("homopolymer", n=3, length=400, seed=5)
    ref = oracle.cross(te[0], te[1], tr[0], tr[1], 9, 5)
    with pkg.gakco_create(4, 9, 5) as ctx:
        out = ctx.cross(te, tr)
    np.testing.assert_array_equal(out["K"], ref["K"])
    assert _close(out["Khat"], ref["Khat"])


def test_refit_replaces_the_training_set():
    tr1 = synth.random_small(94, 30, 4, 20, 100)
    tr2 = synth.random_small(95, 45, 4, 20, 100)
    te = synth.random_small(96, 5, 4, 20, 100)
    with pkg.gakco_create(4, 6, 3) as ctx:
        ctx.cross(te, tr1)
        out = ctx.cross(te, tr2)
    ref = oracle.cross(te[0], te[1], tr2[0], tr2[1], 6, 3)
    np.testing.assert_array_equal(out["K"], ref["K"])


def test_served_requests_equal_their_results_alone():
    """Continuous batching: requests submitted together run in shared
    micro-batches across slots, yet each request's rows equal the result
    of running it alone."""
    tr = synth.random_small(97, 80, 20, 20, 300)
    reqs = [synth.random_small(200 + i, int(n), 20, 0, 300)
            for i, n in enumerate([1, 7, 3, 30, 2, 15, 1, 9, 22, 4, 11, 6])]
    with pkg.gakco_create(20, 8, 4) as ctx:
        ctx.set_option("serve_slots", 2)
        ctx.set_option("serve_max_seqs", 24)  # forces several micro-batches
        ctx.fit(*tr)
        alone = [ctx.cross_fitted(*r) for r in reqs]
        tickets = [ctx.submit(*r) for r in reqs]
        mixed = [ctx.poll(t, timeout_ms=-1) for t in tickets]
        assert ctx.get_stat("served_requests") == len(reqs)
        assert ctx.get_stat("served_batches") >= 2
    for a, m in zip(alone, mixed):
        np.testing.assert_array_equal(m["K"], a["K"])
        np.testing.assert_array_equal(m["Khat"], a["Khat"])
        assert m["latency_ms"] >= 0.0
    r = reqs[3]
    ref = oracle.cross(r[0], r[1], tr[0], tr[1], 8, 4)
    np.testing.assert_array_equal(mixed[3]["K"], ref["K"])


def test_serving_under_a_memory_budget():
    tr = synth.random_small(98, 40, 4, 50, 200)
    reqs = [synth.random_small(300 + i, 5, 4, 50, 200) for i in range(8)]
    with pkg.gakco_create(4, 7, 5) as ctx:
        ctx.set_option("serve_slots", 3)
        ctx.set_option("serve_mem_bytes", 1)  # one batch at a time
        ctx.set_option("serve_max_seqs", 5)
        ctx.fit(*tr)
        tickets = [ctx.submit(*r) for r in reqs]
        outs = [ctx.poll(t, timeout_ms=-1) for t in tickets]
    for r, o in zip(reqs, outs):
        ref = oracle.cross(r[0], r[1], tr[0], tr[1], 7, 5)
        np.testing.assert_array_equal(o["K"], ref["K"])


def test_serving_errors():
    te = synth.random_small(99, 3, 4, 20, 60)
    with pkg.gakco_create(4, 6, 3) as ctx:
        with pytest.raises(pkg.GakcoError):
            ctx.submit(*te)             # no training set yet
        with pytest.raises(pkg.GakcoError):
            ctx.cross_fitted(*te)
        ctx.fit(*synth.random_small(100, 10, 4, 20, 60))
        with pytest.raises(pkg.GakcoError):
            ctx.poll(12345)             # unknown ticket
        bad = te[0].copy()
        bad[0] = 7
        t = ctx.submit(bad, te[1])
        with pytest.raises(pkg.GakcoError) as ei:
            ctx.poll(t, timeout_ms=-1)
        assert ei.value.name == "GAKCO_E_INVALID"
        ok = ctx.poll(ctx.submit(*te), timeout_ms=-1)   # context still serves
        assert ok["K"].shape == (3, 10)


def test_cross_device_api():
    import torch

    tr = synth.random_small(101, 50, 20, 30, 200)
    te = synth.random_small(102, 8, 20, 30, 200)
    dev = torch.device("cuda:0")
    d_tr = torch.from_numpy(tr[0]).to(dev)
    d_te = torch.from_numpy(te[0]).to(dev)
    K = torch.empty((8, 50), dtype=torch.int32, device=dev)
    Kh = torch.empty((8, 50), dtype=torch.float64, device=dev)
    s = torch.cuda.Stream()
    with pkg.gakco_create(20, 8, 4) as ctx:
        ctx.fit_device(d_tr.data_ptr(), tr[1], stream=s.cuda_stream)
        ctx.cross_fitted_device(d_te.data_ptr(), te[1], K.data_ptr(), Kh.data_ptr(),
                                stream=s.cuda_stream)
    s.synchronize()
    ref = oracle.cross(te[0], te[1], tr[0], tr[1], 8, 4)
    np.testing.assert_array_equal(K.cpu().numpy(), ref["K"])
    assert _close(Kh.cpu().numpy(), ref["Khat"])


def test_protein_serving_full_size_sampled():
    """The serving workload's shapes: the N = 3312 protein training set and
    requests of 1-256 protein sequences; sampled rows against the oracle."""
    tr = synth.protein()
    reqs = synth.serve_requests(4, seed=9)
    with pkg.gakco_create(20, 8, 4) as ctx:
        ctx.fit(*tr)
        tickets = [ctx.submit(c, o) for _, c, o in reqs]
        outs = [ctx.poll(t, timeout_ms=-1) for t in tickets]
    for (_, c, o), out in zip(reqs, outs):
        nt = len(o) - 1
        rows = np.unique(np.array([0, nt - 1, nt // 2], dtype=np.int32))
        ref = oracle.cross(c, o, tr[0], tr[1], 8, 4, rows=rows, threads=len(rows))
        np.testing.assert_array_equal(out["K"][rows], ref["K"])
        assert _close(out["Khat"][rows], ref["Khat"])


def test_sequence_window_limit_on_the_cross_path():
    """Counts and window positions are 16-bit fields: a test sequence with
    more than 65535 windows is rejected even where the int32 bound (which
    multiplies by the short training sequences) would allow it."""
    tr = synth.pack([np.zeros(6, np.uint8), np.ones(7, np.uint8)])
    te = synth.pack([np.zeros(70000, np.uint8)])
    with pkg.gakco_create(4, 4, 3) as ctx:
        ctx.fit(*tr)
        with pytest.raises(pkg.GakcoError) as ei:
            ctx.cross_fitted(*te)
        assert ei.value.name == "GAKCO_E_OVERFLOW"
        ok = ctx.cross_fitted(*synth.pack([np.zeros(60, np.uint8)]))
        assert ok["K"].shape == (1, 2)


def test_gram_after_fit_and_cross_on_one_context():
    """A Gram call's cached graph must not be replayed after fit and cross
    calls on the same context rewrote its tables and buffers: the repeated
    Gram call plans again and stays exact."""
    a = synth.random_small(110, 60, 4, 50, 250)
    b = synth.random_small(111, 140, 4, 50, 300)
    with pkg.gakco_create(4, 8, 5) as ctx:
        ctx.set_option("dense", 1)
        first = ctx.gram(*a, khat=True)
        ctx.fit(*b)
        ctx.cross_fitted(*a)
        again = ctx.gram(*a, khat=True)
        assert ctx.get_stat("graph_replay") == 0
        ctx.extend(*synth.random_small(112, 9, 4, 50, 250))
        third = ctx.gram(*a, khat=True)
    ref = oracle.gram(*a, 8, 5)
    for out in (first, again, third):
        np.testing.assert_array_equal(out["K"], ref["K"])
        assert _close(out["Khat"], ref["Khat"])
