"""Parity of the CUDA engine with the CPU oracle, through the C ABI.

Integer outputs (K and every N_m) must be bit-exact; the normalised kernel
must agree within 1e-12 relative (both sides compute it in fp64, the engine
as (K * r_x) * r_y with r = 1/sqrt(K(x, x)), a few ulp from the oracle's
K / sqrt(Kxx Kyy)).
"""

import math

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
    pkg.load_library()


def _check(out, ref, rows=None, nm=True):
    K = out["K"] if rows is None else out["K"][rows]
    np.testing.assert_array_equal(K, ref["K"])
    if nm:
        Nm = out["Nm"] if rows is None else out["Nm"][:, rows]
        np.testing.assert_array_equal(Nm, ref["Nm"])
    Kh = out["Khat"] if rows is None else out["Khat"][rows]
    err = np.abs(Kh - ref["Khat"])
    assert np.all(err <= KHAT_RTOL * np.maximum(np.abs(ref["Khat"]), 1e-300) + 1e-300), \
        f"max Khat err {err.max()}"


def _gram(sigma, g, k, codes, off, **opts):
    with pkg.gakco_create(sigma, g, k) as ctx:
        for name, v in opts.items():
            ctx.set_option(name, v)
        return ctx.gram(codes, off, khat=True, nm=True)


@pytest.mark.parametrize("engine", [0, 1])
def test_dna_toy_bit_exact(engine):
    codes, off = synth.dna_toy()
    ref = oracle.gram(codes, off, 7, 5)
    _check(_gram(4, 7, 5, codes, off, engine=engine), ref)


RAGGED = [  # (seed, n, sigma, lo, hi, g, k)
    (20, 37, 4, 0, 260, 6, 3),      # empty and short sequences, several tiles
    (21, 64, 20, 0, 400, 8, 4),     # protein alphabet, 40-bit keys
    (22, 50, 36, 5, 300, 8, 5),     # text alphabet, 48-bit keys (wide sort)
    (23, 20, 4, 8, 120, 10, 6),     # DNA g = 10, M = 4
    (24, 9, 2, 0, 50, 3, 1),        # binary alphabet, M = 2
    (25, 15, 5, 1, 90, 5, 5),       # k = g: spectrum kernel, M = 0
    (26, 12, 3, 2, 60, 9, 1),       # M = 8: nine levels
]


@pytest.mark.parametrize("case", RAGGED)
@pytest.mark.parametrize("engine", [0, 1])
def test_ragged_random_bit_exact(case, engine):
    seed, n, sigma, lo, hi, g, k = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    ref = oracle.gram(codes, off, g, k)
    _check(_gram(sigma, g, k, codes, off, engine=engine), ref)


NSWEEP = [  # (name, sigma, g, k, n): the N-sweep at l = 100 (Section 3.2, Fig. 5(c))
    ("dna_sigma5", 5, 10, 6, 100),   # DNA with the unknown-base symbol N (Section S:3.2)
    ("dna_sigma5", 5, 10, 6, 750),
    ("protein", 20, 8, 4, 250),
    ("text", 36, 8, 5, 250),
]


@pytest.mark.parametrize("case", NSWEEP, ids=[f"{c[0]}_{c[4]}" for c in NSWEEP])
def test_nsweep_configurations_bit_exact(case):
    """The sweep's own inputs and options (the cost model picks the dense
    levels), every entry against the oracle."""
    name, sigma, g, k, n = case
    codes, off = synth.fixed_length(1000 + n, n, 100, sigma)
    ref = oracle.gram(codes, off, g, k)
    _check(_gram(sigma, g, k, codes, off, dense=1), ref)


@pytest.mark.parametrize("opts", [
    {"radix_bits": 4}, {"radix_bits": 11}, {"chunk_elems": 4096},
    {"smem_cols": 7}, {"smem_cols": 32, "accum_threads": 256},
    {"accum_threads": 1024}, {"graph": 0},
    {"accum_variant": 1}, {"accum_variant": 2}, {"accum_variant": 1, "accum_threads": 512},
    {"accum_variant": 2, "smem_cols": 32}, {"rle_items": 8}, {"rle_items": 8, "chunk_elems": 4096},
    {"level_radix_bits": (2 << 8) | 11}, {"level_radix_bits": (4 << 8) | 5},
])
def test_tuning_options_do_not_change_results(opts):
    codes, off = synth.random_small(30, 70, 20, 0, 300)
    ref = oracle.gram(codes, off, 8, 4)
    _check(_gram(20, 8, 4, codes, off, **opts), ref)


SORT_CASES = [  # (seed, n, sigma, lo, hi, g, k, options): the onesweep sort
    (40, 70, 20, 0, 300, 8, 4, {}),                       # protein alphabet, 31-bit folded keys
    (41, 50, 36, 5, 300, 8, 5, {}),                       # text, 64-bit keys (wide)
    (42, 60, 4, 0, 260, 10, 6, {"radix_bits": 6}),        # 6-bit digits, 3-4 passes
    (43, 40, 4, 50, 200, 10, 6, {"chunk_elems": 4096}),   # one tile per chunk: many chunks and epochs
    (44, 300, 4, 100, 300, 10, 6, {"chunk_elems": 1 << 16}),  # many tiles per segment: long look-backs
    (45, 20, 5, 1, 90, 5, 5, {}),                         # M = 0
    (46, 30, 4, 0, 200, 8, 4, {"radix_bits": 11}),        # wider digits: the classic sort runs
]


@pytest.mark.parametrize("case", SORT_CASES)
@pytest.mark.parametrize("engine", [0, 1])
def test_onesweep_sort_bit_exact(case, engine):
    seed, n, sigma, lo, hi, g, k, opts = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    ref = oracle.gram(codes, off, g, k)
    _check(_gram(sigma, g, k, codes, off, sort=1, engine=engine, **opts), ref)


def test_onesweep_fit_cross_and_graph_replay():
    """The fitted index and the cross kernel sort through the same path;
    a replayed Gram graph clears and renumbers the look-back words."""
    codes, off = synth.random_small(47, 120, 20, 20, 400)
    tcodes, toff = synth.random_small(48, 17, 20, 0, 300)
    ref = oracle.gram(codes, off, 8, 4)
    xref = oracle.cross(tcodes, toff, codes, off, 8, 4)
    with pkg.gakco_create(20, 8, 4) as ctx:
        ctx.set_option("sort", 1)
        a = ctx.gram(codes, off, khat=True, nm=True)
        b = ctx.gram(codes, off, khat=True, nm=True)
        ctx.fit(codes, off)
        x = ctx.cross_fitted(tcodes, toff, khat=True)
    _check(a, ref)
    _check(b, ref)
    np.testing.assert_array_equal(x["K"], xref["K"])


@pytest.mark.parametrize("case", RAGGED)
def test_run_length_with_eight_items_per_thread(case):
    seed, n, sigma, lo, hi, g, k = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    ref = oracle.gram(codes, off, g, k)
    _check(_gram(sigma, g, k, codes, off, rle_items=8), ref)


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("case", RAGGED[:4])
def test_accumulation_variants_bit_exact(case, variant):
    seed, n, sigma, lo, hi, g, k = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    ref = oracle.gram(codes, off, g, k)
    _check(_gram(sigma, g, k, codes, off, accum_variant=variant), ref)


def test_caller_kept_outputs_are_rewritten_in_place():
    """gram_batch(out=...) writes every call's results into the given host
    arrays (returned as the same objects); a wrong shape or dtype is
    refused before the call."""
    sets = [synth.random_small(31, 40, 4, 50, 200), synth.random_small(32, 25, 4, 50, 200)]
    refs = [oracle.gram(c, o, 10, 6) for c, o in sets]
    outs = [{"K": np.full((len(o) - 1, len(o) - 1), -1, np.int32),
             "Khat": np.full((len(o) - 1, len(o) - 1), np.nan)} for _, o in sets]
    with pkg.gakco_create(4, 10, 6) as ctx:
        for _ in range(2):
            got = ctx.gram_batch(sets, khat=True, nm=False, out=outs)
            assert got is outs
            for out, ref in zip(outs, refs):
                _check(out, ref, nm=False)
            for out in outs:
                out["K"].fill(-1)
                out["Khat"].fill(np.nan)
        bad = [{"K": np.empty((3, 3), np.int32), "Khat": outs[0]["Khat"]}, outs[1]]
        with pytest.raises(ValueError):
            ctx.gram_batch(sets, khat=True, out=bad)
        with pytest.raises(ValueError):
            ctx.gram_batch(sets, khat=True, out=[{"K": outs[0]["K"], "Khat": outs[0]["Khat"].astype(np.float32)},
                                                 outs[1]])


@pytest.mark.parametrize("kind", ["homopolymer", "period2", "mixed"])
def test_repetitive_sequences_large_counts(kind):
    """Counts of one feature in one sequence far above 127."""
    codes, off = synth.repeats(kind, n=5, length=700)
    ref = oracle.gram(codes, off, 10, 6)
    _check(_gram(4, 10, 6, codes, off), ref)


def test_batch_equals_individual_calls():
    sets = [synth.random_small(40 + i, n, 4, 50, 200) for i, n in enumerate([30, 1, 0, 45])]
    with pkg.gakco_create(4, 8, 5) as ctx:
        batch = ctx.gram_batch(sets, khat=True, nm=True)
        for (c, o), b in zip(sets, batch):
            single = ctx.gram(c, o, khat=True, nm=True)
            for key in ("K", "Nm", "Khat"):
                np.testing.assert_array_equal(b[key], single[key])
            if len(o) > 1:
                ref = oracle.gram(c, o, 8, 5)
                _check(b, ref)


def test_graph_replay_is_used_and_identical():
    codes, off = synth.random_small(50, 40, 4, 20, 150)
    with pkg.gakco_create(4, 7, 4) as ctx:
        a = ctx.gram(codes, off, khat=True, nm=True)
        assert ctx.get_stat("graph_replay") == 0
        b = ctx.gram(codes, off, khat=True, nm=True)
        assert ctx.get_stat("graph_replay") == 1
        for key in ("K", "Nm", "Khat"):
            np.testing.assert_array_equal(a[key], b[key])
        assert ctx.get_stat("launches") > 0


def test_degenerate_inputs():
    g, k = 5, 3
    cases = [
        synth.pack([]),                                  # no sequences
        synth.pack([np.zeros(3, np.uint8)]),             # one sequence, no window
        synth.pack([np.zeros(5, np.uint8)]),             # exactly one window
        synth.pack([np.array([], np.uint8)] * 3),        # empty sequences only
    ]
    with pkg.gakco_create(4, g, k) as ctx:
        for codes, off in cases:
            out = ctx.gram(codes, off, khat=True, nm=True)
            n = len(off) - 1
            if n:
                ref = oracle.gram(codes, off, g, k)
                _check(out, ref)
            else:
                assert out["K"].shape == (0, 0)


def test_invalid_symbol_is_rejected_and_context_survives():
    codes, off = synth.random_small(60, 6, 4, 10, 40)
    bad = codes.copy()
    bad[5] = 4
    with pkg.gakco_create(4, 5, 3) as ctx:
        with pytest.raises(pkg.GakcoError) as ei:
            ctx.gram(bad, off)
        assert ei.value.name == "GAKCO_E_INVALID"
        _check(ctx.gram(codes, off, khat=True, nm=True), oracle.gram(codes, off, 5, 3))


def test_overflow_bound_is_enforced():
    # C(10, 4) * W^2 >= 2^31 for W = 3200.
    codes, off = synth.pack([np.zeros(3209, np.uint8)])
    with pkg.gakco_create(4, 10, 6) as ctx:
        with pytest.raises(pkg.GakcoError) as ei:
            ctx.gram(codes, off)
        assert ei.value.name == "GAKCO_E_OVERFLOW"


def test_injected_allocation_failure_leaves_context_usable():
    codes, off = synth.random_small(61, 10, 4, 10, 60)
    with pkg.gakco_create(4, 6, 3) as ctx:
        ctx.set_option("fail_alloc_after", 1)
        with pytest.raises(pkg.GakcoError) as ei:
            ctx.gram(codes, off)
        assert ei.value.name == "GAKCO_E_OOM"
        _check(ctx.gram(codes, off, khat=True, nm=True), oracle.gram(codes, off, 6, 3))


def test_device_api_with_torch_buffers_and_stream():
    import torch

    codes, off = synth.random_small(62, 33, 20, 30, 200)
    g, k = 8, 4
    n = len(off) - 1
    dev = torch.device("cuda:0")
    d_codes = torch.from_numpy(codes).to(dev)
    K = torch.empty((n, n), dtype=torch.int32, device=dev)
    Kh = torch.empty((n, n), dtype=torch.float64, device=dev)
    Nm = torch.empty((g - k + 1, n, n), dtype=torch.int32, device=dev)
    s = torch.cuda.Stream()
    with pkg.gakco_create(20, g, k) as ctx:
        ctx.gram_device(d_codes.data_ptr(), off, K.data_ptr(), Kh.data_ptr(),
                        Nm.data_ptr(), stream=s.cuda_stream)
    s.synchronize()
    ref = oracle.gram(codes, off, g, k)
    _check({"K": K.cpu().numpy(), "Nm": Nm.cpu().numpy(), "Khat": Kh.cpu().numpy()}, ref)


def test_autotune_keeps_results_and_caches_its_choice():
    import torch

    sets = [synth.random_small(64 + i, n, 4, 80, 200) for i, n in enumerate([60, 90])]
    dev = torch.device("cuda:0")
    d_codes = [torch.from_numpy(c).to(dev) for c, _ in sets]
    with pkg.gakco_create(4, 8, 5) as ctx:
        rep = ctx.autotune_device([t.data_ptr() for t in d_codes], [o for _, o in sets])
        assert "radix_bits=" in rep or rep == "cached"
        outs = ctx.gram_batch(sets, khat=True, nm=True)
    with pkg.gakco_create(4, 8, 5) as ctx:
        assert ctx.autotune_device([t.data_ptr() for t in d_codes], [o for _, o in sets]) == "cached"
    for (c, o), out in zip(sets, outs):
        _check(out, oracle.gram(c, o, 8, 5))


def test_work_statistics_follow_their_definitions():
    """Packing reads every symbol once and writes a key and a window id per
    window; the combine tail reads the upper triangles of C_0..C_M once and
    writes every requested output; every stage with work reports bytes."""
    g, k = 8, 4
    codes, off = synth.random_small(60, 45, 20, 0, 300)
    n, M = len(off) - 1, g - k
    G = int(np.maximum(np.diff(off) - g + 1, 0).sum())
    with pkg.gakco_create(20, g, k) as ctx:
        ctx.gram(codes, off, khat=True, nm=True)
        assert ctx.get_stat("pack_bytes") == float(off[-1] + 12 * G)
        assert ctx.get_stat("combine_bytes") == 4.0 * (M + 1) * n * (n + 1) / 2 + (4 + 8 + 4 * (M + 1)) * n * n
        assert ctx.get_stat("sort_bytes") > 0 and ctx.get_stat("rle_bytes") > 0
        assert ctx.get_stat("masks") == sum(math.comb(g, m) for m in range(M + 1))


def test_shared_atomic_probe_rates():
    a = pkg.gakco_measure_smem_atomics()
    r = pkg.gakco_measure_smem_atomics(random_columns=True)
    assert a > 1e11 and r > 1e10
    assert r <= 1.05 * a
