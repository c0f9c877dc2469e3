"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test checks the brute-force oracle against something the paper or the
mathematics fixes: the worked example printed with Fig. 2, the gapped k-mer
feature-map definition (Eq. 4) enumerated explicitly, the paper's own
mask-and-count route (Eq. 8 and Eq. 9) restated with dictionaries, the
spectrum-kernel special case (Eq. 3), and invariants that hold for any
input.  A plausible slip in the oracle (a window too many or too few, a
wrong h_m, a dropped self pair, transposed operands) fails at least one.
"""

import itertools
import os
from collections import Counter
from math import comb

import numpy as np
import pytest

import oracle
from paper_1704_07468_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DNA = {"A": 0, "C": 1, "G": 2, "T": 3}


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = vals
    return out


def _encode(strings):
    return synth.pack([np.array([DNA[c] for c in s], dtype=np.uint8)
                       for s in strings])


def _seqs(codes, offsets):
    return [codes[offsets[i]:offsets[i + 1]] for i in range(len(offsets) - 1)]


def _windows(seq, g):
    return [tuple(int(c) for c in seq[i:i + g]) for i in range(len(seq) - g + 1)]


# ---------------------------------------------------------------- Fig. 2 ----

def test_fig2_worked_example():
    """Fig. 2 caption: S = ACACA, T = AAACA, g = 3 gives N_0(S,T) = 2,
    C_1(S,T) = 9 and N_1(S,T) = 3."""
    gold = _read_golden("fig2_worked_example.txt")
    g = int(gold["g"][0])
    codes, off = _encode([gold["S"][0], gold["T"][0]])
    nm = oracle.mismatch_profile(codes, off, g, g)
    assert nm[0, 0, 1] == int(gold["N0_ST"][0])
    assert nm[1, 0, 1] == int(gold["N1_ST"][0])
    # Eq. 8 with the printed numbers: C_1 = N_1 + C(g, 1) N_0.
    assert nm[1, 0, 1] + comb(g, 1) * nm[0, 0, 1] == int(gold["C1_ST"][0])
    # The caption's g-mer lists: three windows each, nine pairs in total.
    assert len(gold["gmers_S"]) * len(gold["gmers_T"]) == nm[:, 0, 1].sum()


def test_fig2_windows_are_contiguous_substrings():
    """The caption lists the g-mers of S and T as the contiguous windows."""
    gold = _read_golden("fig2_worked_example.txt")
    g = int(gold["g"][0])
    for name in ("S", "T"):
        s = gold[name][0]
        assert [s[i:i + g] for i in range(len(s) - g + 1)] == gold["gmers_" + name]


def test_fig2_kernel_values_by_hand():
    """K(S,T) from Eq. 6/7 with the caption's counts: k=2 gives h=[3,1] and
    K = 3*2 + 1*3 = 9; k=1 gives h=[3,2,1], N_2 = 3 and K = 6+6+3 = 15."""
    codes, off = _encode(["ACACA", "AAACA"])
    assert oracle.gram(codes, off, 3, 2)["K"][0, 1] == 9
    assert oracle.gram(codes, off, 3, 1)["K"][0, 1] == 15


# ------------------------------------------------ Eq. 4 feature enumeration --

def _gapped_kmer_counts(seq, g, k):
    """Explicit gapped k-mer features of Eq. 4: every g-mer contributes one
    feature per choice of k of its g positions, identified by the chosen
    positions and the symbols found there."""
    c = Counter()
    for w in _windows(seq, g):
        for pos in itertools.combinations(range(g), k):
            c[(pos, tuple(w[p] for p in pos))] += 1
    return c


def _eq4_kernel(seqs, g, k):
    feats = [_gapped_kmer_counts(s, g, k) for s in seqs]
    n = len(seqs)
    K = np.zeros((n, n), dtype=np.int64)
    for x in range(n):
        for y in range(n):
            K[x, y] = sum(v * feats[y].get(f, 0) for f, v in feats[x].items())
    return K


CASES = [  # (seed, n, sigma, lo, hi, g)
    (0, 5, 2, 0, 9, 3), (1, 4, 3, 2, 10, 4), (2, 6, 4, 0, 12, 5),
    (3, 3, 4, 5, 12, 6), (4, 5, 2, 1, 8, 1), (5, 4, 3, 3, 11, 2),
]


@pytest.mark.parametrize("case", CASES)
def test_eq4_enumeration_equals_oracle(case):
    seed, n, sigma, lo, hi, g = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    seqs = _seqs(codes, off)
    for k in range(1, g + 1):
        K = oracle.gram(codes, off, g, k)["K"]
        np.testing.assert_array_equal(K, _eq4_kernel(seqs, g, k),
                                      err_msg=f"g={g} k={k}")


# ------------------------------------- Eq. 8 / Eq. 9: mask-and-count route --

def _cumulative_profiles(seqs, g, M):
    """C_m(x, y) for m = 0..M by the route of Section 2.2 (Fig. 2, steps
    3-5): for each of the C(g, m) position sets, delete those positions from
    every g-mer, count each remaining (g-m)-mer per sequence, and add
    c_x * c_y over shared (g-m)-mers."""
    n = len(seqs)
    C = np.zeros((M + 1, n, n), dtype=np.int64)
    for m in range(M + 1):
        for dele in itertools.combinations(range(g), m):
            keep = [p for p in range(g) if p not in dele]
            cnt = [Counter(tuple(w[p] for p in keep) for w in _windows(s, g))
                   for s in seqs]
            for x in range(n):
                for y in range(n):
                    C[m, x, y] += sum(v * cnt[y].get(f, 0)
                                      for f, v in cnt[x].items())
    return C


def _inclusion_exclusion(C, g):
    """Eq. 9: N_m = C_m - sum_{j<m} C(g-j, m-j) N_j."""
    N = np.zeros_like(C)
    for m in range(C.shape[0]):
        N[m] = C[m] - sum(comb(g - j, m - j) * N[j] for j in range(m))
    return N


@pytest.mark.parametrize("case", CASES[:4])
def test_mask_counting_route_equals_oracle(case):
    seed, n, sigma, lo, hi, g = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    seqs = _seqs(codes, off)
    M = g - 1 if g > 1 else 0
    C = _cumulative_profiles(seqs, g, M)
    nm = oracle.mismatch_profile(codes, off, g, M)
    np.testing.assert_array_equal(_inclusion_exclusion(C, g), nm)
    # Eq. 8 in the forward direction.
    for m in range(M + 1):
        fwd = nm[m] + sum(comb(g - j, m - j) * nm[j] for j in range(m))
        np.testing.assert_array_equal(fwd, C[m])


@pytest.mark.parametrize("case", CASES[:4])
def test_oracle_counting_route_equals_brute_force(case):
    """The oracle's own per-mask counting route (used to check sharded
    computations) against its brute-force Hamming histogram, through Eq. 9,
    and summed over any split of the masks."""
    seed, n, sigma, lo, hi, g = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    M = g - 1 if g > 1 else 0
    masks = oracle.position_masks(g, M)
    assert len(masks) == sum(comb(g, m) for m in range(M + 1))
    assert masks == sorted(masks, key=lambda d: (len(d), d))
    C = oracle.cumulative_profile(codes, off, g, M)
    np.testing.assert_array_equal(oracle.inclusion_exclusion(C, g),
                                  oracle.mismatch_profile(codes, off, g, M))
    cut = len(masks) // 3
    parts = (oracle.cumulative_profile(codes, off, g, M, masks[:cut])
             + oracle.cumulative_profile(codes, off, g, M, masks[cut:]))
    np.testing.assert_array_equal(parts, C)


@pytest.mark.parametrize("case", CASES[:4])
def test_kernel_equals_top_level_cumulative_profile(case):
    """sum_m C(g-m, k) N_m equals C_M with M = g - k, because C(g-m, k) =
    C(g-m, M-m) is the coefficient of N_m in Eq. 8 at level M."""
    seed, n, sigma, lo, hi, g = case
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    seqs = _seqs(codes, off)
    for k in range(1, g + 1):
        M = g - k
        C = _cumulative_profiles(seqs, g, M)
        np.testing.assert_array_equal(oracle.gram(codes, off, g, k)["K"], C[M])


# ------------------------------------------------- Eq. 3: spectrum case ----

def test_spectrum_special_case():
    """k = g (no gaps): K is the spectrum kernel of Eq. 3 on g-mers."""
    codes, off = synth.random_small(7, 8, 3, 0, 30)
    seqs = _seqs(codes, off)
    for g in (1, 2, 3, 4):
        cnt = [Counter(_windows(s, g)) for s in seqs]
        ref = np.array([[sum(v * b.get(f, 0) for f, v in a.items())
                         for b in cnt] for a in cnt])
        np.testing.assert_array_equal(oracle.gram(codes, off, g, g)["K"], ref)


# ------------------------------------------------------------ invariants ----

def test_profile_sums_to_all_window_pairs():
    """Histogramming every distance 0..g counts every window pair once."""
    codes, off = synth.random_small(8, 7, 4, 0, 40)
    lens = np.diff(off)
    for g in (1, 3, 6):
        nm = oracle.mismatch_profile(codes, off, g, g)
        W = np.maximum(lens - g + 1, 0)
        np.testing.assert_array_equal(nm.sum(axis=0), np.outer(W, W))


def test_symmetry_and_self_matches():
    codes, off = synth.random_small(9, 9, 3, 0, 50)
    seqs = _seqs(codes, off)
    g, k = 5, 3
    nm = oracle.mismatch_profile(codes, off, g, g - k)
    for m in range(nm.shape[0]):
        np.testing.assert_array_equal(nm[m], nm[m].T)
    # N_0(x, x) = sum over distinct g-mers of (count)^2, which is >= W_x.
    for x, s in enumerate(seqs):
        c = Counter(_windows(s, g))
        assert nm[0, x, x] == sum(v * v for v in c.values())
        assert nm[0, x, x] >= max(len(s) - g + 1, 0)


def test_gram_is_positive_semidefinite():
    """K is an inner product of feature counts (Eq. 2), hence PSD."""
    codes, off = synth.random_small(10, 24, 4, 20, 60)
    K = oracle.gram(codes, off, 6, 3)["K"].astype(np.float64)
    ev = np.linalg.eigvalsh(K)
    assert ev.min() >= -1e-9 * np.abs(K).max()


def test_normalised_kernel_properties():
    codes, off = synth.pack([np.zeros(2, np.uint8), np.arange(20) % 3,
                             np.arange(30) % 2, np.array([], np.uint8)])
    res = oracle.gram(codes, off, 4, 2)
    Kh = res["Khat"]
    W = np.maximum(np.diff(off) - 4 + 1, 0)
    for x in range(len(W)):
        assert Kh[x, x] == (1.0 if W[x] > 0 else 0.0)
    assert np.all(np.abs(Kh) <= 1.0 + 1e-15)
    assert np.all(Kh[W == 0] == 0.0) and np.all(Kh[:, W == 0] == 0.0)
    assert not np.any(np.isnan(Kh))


def test_hamming_deletion_property_s11():
    """Section S:1.1: equal after deleting p positions implies distance <= p,
    and conversely every pair at distance d <= p is equal after deleting
    exactly the C(g-d, p-d) position sets that cover its mismatches."""
    rng = np.random.default_rng(12)
    g = 6
    for _ in range(300):
        a = rng.integers(0, 2, g)
        b = rng.integers(0, 2, g)
        d = int((a != b).sum())
        for p in range(g + 1):
            equal_sets = 0
            for dele in itertools.combinations(range(g), p):
                keep = [i for i in range(g) if i not in dele]
                if np.array_equal(a[keep], b[keep]):
                    equal_sets += 1
                    assert d <= p
            assert equal_sets == (comb(g - d, p - d) if d <= p else 0)


# ------------------------------------------------------ oracle's own API ----

def test_sampled_rows_and_self_profile_agree_with_full():
    codes, off = synth.random_small(13, 10, 4, 0, 45)
    g, M = 5, 2
    full = oracle.mismatch_profile(codes, off, g, M)
    rows = np.array([7, 0, 3])
    np.testing.assert_array_equal(
        oracle.mismatch_profile(codes, off, g, M, rows=rows), full[:, rows])
    sp = oracle.self_profile(codes, off, g, M)
    np.testing.assert_array_equal(sp, np.stack([np.diag(p) for p in full]))


def test_cross_is_a_block_of_the_joint_gram():
    """The paper computes one kernel over train and test together (Section
    3.1); the cross kernel is the test-rows x train-columns block of it."""
    tr_c, tr_o = synth.random_small(14, 6, 4, 0, 40)
    te_c, te_o = synth.random_small(15, 4, 4, 0, 40)
    g, k = 5, 3
    both_c = np.concatenate([tr_c, te_c])
    both_o = np.concatenate([tr_o, te_o[1:] + tr_o[-1]])
    joint = oracle.gram(both_c, both_o, g, k)
    cr = oracle.cross(te_c, te_o, tr_c, tr_o, g, k)
    np.testing.assert_array_equal(cr["K"], joint["K"][6:, :6])
    np.testing.assert_array_equal(cr["Khat"], joint["Khat"][6:, :6])


def test_planted_mistakes_are_caught(monkeypatch):
    """A wrong h_m (C(g, m) in place of C(g-m, k)) planted in the oracle
    fails the Eq. 4 pin."""
    seed, n, sigma, lo, hi, g = CASES[2]
    codes, off = synth.random_small(seed, n, sigma, lo, hi)
    ref = _eq4_kernel(_seqs(codes, off), g, 3)
    monkeypatch.setattr(oracle, "h_coefficients",
                        lambda g_, k_: np.array([comb(g_, m) for m in range(g_ - k_ + 1)]))
    assert not np.array_equal(oracle.gram(codes, off, g, 3)["K"], ref)


def test_planted_window_off_by_one_is_caught():
    """Dropping the last window of every sequence (l - g windows instead of
    l - g + 1) breaks the total-pairs invariant."""
    codes, off = synth.random_small(16, 5, 3, 4, 20)
    g = 3
    trimmed_codes = np.concatenate([codes[off[i]:off[i + 1] - 1]
                                    for i in range(len(off) - 1)])
    trimmed_off = off - np.arange(len(off))
    nm = oracle.mismatch_profile(trimmed_codes, trimmed_off, g, g)
    W = np.maximum(np.diff(off) - g + 1, 0)
    assert not np.array_equal(nm.sum(axis=0), np.outer(W, W))
