"""Seeded synthetic sequence datasets.

This module only draws random sequences; it holds none of the kernel's
arithmetic.  Both the CUDA path and the CPU oracle are fed from here, so a
dataset is always the same bytes on both sides.

A dataset is a pair ``(codes, offsets)``:

* ``codes``   -- ``uint8`` array, all sequences concatenated, each symbol a
  code in ``[0, sigma)``;
* ``offsets`` -- ``int64`` array of length ``n + 1``; sequence ``x`` is
  ``codes[offsets[x]:offsets[x + 1]]``.

The workloads follow the shapes of the paper's benchmark tasks (Table 3 and
Section S:3.2): DNA binding-site sets (N = 4000, length 100), SCOP protein
sets (N = 3312, lengths up to about 1000, alphabet of 20 residues) and
character text (alphabet of 36).  The real datasets are not used; these
generators stand in for them.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "pack",
    "dna_toy",
    "dna_large",
    "protein",
    "text",
    "serve_requests",
    "repeats",
    "periodic",
    "fixed_length",
    "random_small",
    "WORKLOADS",
]


def pack(seqs):
    """Concatenate a list of uint8 arrays into ``(codes, offsets)``."""
    seqs = [np.asarray(s, dtype=np.uint8) for s in seqs]
    lens = np.array([len(s) for s in seqs], dtype=np.int64)
    offsets = np.zeros(len(seqs) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    codes = np.concatenate(seqs) if seqs else np.zeros(0, dtype=np.uint8)
    return np.ascontiguousarray(codes, dtype=np.uint8), offsets


def _draw(rng, lengths, probs):
    sigma = len(probs)
    total = int(np.sum(lengths))
    codes = rng.choice(sigma, size=total, p=probs).astype(np.uint8)
    offsets = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(np.asarray(lengths, dtype=np.int64), out=offsets[1:])
    return codes, offsets


def dna_toy(seed=1, n=200, length=100):
    """DNA, sigma = 4 (A, C, G, T as codes 0..3), iid uniform, fixed length."""
    rng = np.random.default_rng(seed)
    return _draw(rng, np.full(n, length, dtype=np.int64), np.full(4, 0.25))


# GC content 0.4: P(A) = P(T) = 0.3, P(C) = P(G) = 0.2 (codes A=0, C=1, G=2, T=3).
DNA_GC04 = np.array([0.3, 0.2, 0.2, 0.3])
DNA_LARGE_SIZES = (500, 1000, 2000, 3000, 4000)


def dna_large(seeds=(2, 3, 4, 5, 6), sizes=DNA_LARGE_SIZES, lo=100, hi=300):
    """Five independent DNA datasets of uneven size and length.

    Dataset ``i`` has ``sizes[i]`` sequences with lengths uniform in
    ``[lo, hi]`` and GC content 0.4, drawn with ``seeds[i]``.
    """
    out = []
    for seed, n in zip(seeds, sizes):
        rng = np.random.default_rng(seed)
        lengths = rng.integers(lo, hi + 1, size=n)
        out.append(_draw(rng, lengths, DNA_GC04))
    return out


def protein_law(seed=7):
    """Residue frequencies of the protein workload: Dirichlet(2 * 1_20)."""
    rng = np.random.default_rng(seed)
    return rng, rng.dirichlet(np.full(20, 2.0))


def protein_lengths(rng, n, median=300.0, sigma=0.5, lo=50, hi=1000):
    """Log-normal lengths (median 300, log-sd 0.5), rounded, clipped."""
    raw = rng.lognormal(np.log(median), sigma, size=n)
    return np.clip(np.round(raw), lo, hi).astype(np.int64)


def protein(seed=7, n=3312):
    """Protein, sigma = 20, SCOP-1.34-sized (N = 3312)."""
    rng, probs = protein_law(seed)
    lengths = protein_lengths(rng, n)
    return _draw(rng, lengths, probs)


def text(seed=8, n=6000, lo=200, hi=2000, s=1.1):
    """Character text, sigma = 36, Zipf(s) symbol frequencies by rank."""
    rng = np.random.default_rng(seed)
    probs = np.arange(1, 37, dtype=np.float64) ** (-s)
    probs /= probs.sum()
    lengths = rng.integers(lo, hi + 1, size=n)
    return _draw(rng, lengths, probs)


def serve_requests(n_requests, seed=9, law_seed=7, mean_gap_s=0.005,
                   max_batch=256):
    """Poisson stream of protein test batches.

    Returns a list of ``(arrival_s, codes, offsets)``; inter-arrival gaps are
    exponential with mean ``mean_gap_s``, batch sizes uniform in
    ``[1, max_batch]``, residues drawn from the protein workload's law and
    lengths from its length law.
    """
    _, probs = protein_law(law_seed)
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += rng.exponential(mean_gap_s)
        b = int(rng.integers(1, max_batch + 1))
        lengths = protein_lengths(rng, b)
        codes, offsets = _draw(rng, lengths, probs)
        out.append((t, codes, offsets))
    return out


def repeats(kind="homopolymer", n=4, length=1500, sigma=4, seed=11):
    """Highly repetitive sequences (counts of one feature above 127).

    ``homopolymer``: every symbol equal; ``period2``: alternating pair;
    ``mixed``: some homopolymers, some period-2, some random.
    """
    rng = np.random.default_rng(seed)
    seqs = []
    for i in range(n):
        if kind == "homopolymer" or (kind == "mixed" and i % 3 == 0):
            seqs.append(np.full(length - 7 * i, i % sigma, dtype=np.uint8))
        elif kind == "period2" or (kind == "mixed" and i % 3 == 1):
            a, b = i % sigma, (i + 1) % sigma
            s = np.empty(length - 5 * i, dtype=np.uint8)
            s[0::2] = a
            s[1::2] = b
            seqs.append(s)
        else:
            seqs.append(rng.integers(0, sigma, size=length // 3).astype(np.uint8))
    return pack(seqs)


def periodic(seed, period, lengths, shifts, sigma=4):
    """Sequences cut from one random unit repeated end to end.

    The unit holds ``period`` iid uniform symbols; sequence ``i`` starts at
    position ``shifts[i]`` of the unit and runs on cyclically for
    ``lengths[i]`` symbols, so every window of a sequence recurs once per
    period (counts of a feature near ``length / period``).
    """
    rng = np.random.default_rng(seed)
    unit = rng.integers(0, sigma, size=period).astype(np.uint8)
    seqs = []
    for length, shift in zip(lengths, shifts):
        idx = (int(shift) + np.arange(int(length))) % period
        seqs.append(unit[idx])
    return pack(seqs)


def fixed_length(seed, n, length, sigma):
    """``n`` sequences of one ``length``, iid uniform over ``sigma`` symbols
    (the N-sweep at l = 100 of Section 3.2 / Fig. 5(c); sigma = 5 is DNA
    with the unknown-base symbol N of Section S:3.2)."""
    rng = np.random.default_rng(seed)
    codes = rng.integers(0, sigma, size=n * length).astype(np.uint8)
    return codes, np.arange(0, n * length + 1, length, dtype=np.int64)


def random_small(seed, n, sigma, lo, hi):
    """Small iid uniform dataset with lengths uniform in ``[lo, hi]``."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(lo, hi + 1, size=n)
    return _draw(rng, lengths, np.full(sigma, 1.0 / sigma))


# name -> (sigma, g, k, builder) for the single-dataset workloads.
WORKLOADS = {
    "dna_toy": (4, 7, 5, dna_toy),
    "protein": (20, 8, 4, protein),
    "text": (36, 8, 5, text),
}
