"""Write the per-row digests of the benchmark-size workloads from the CPU
oracle alone.

For every row x of a dataset the digest is the first 16 hex digits of the
SHA-256 of the little-endian int64 bytes of K[x, :] followed by N_0[x, :],
..., N_M[x, :] (Definition 1, Eq. 7), over all columns.  Rows covered:

* DNA toy (N = 200, g = 7, k = 5): every row;
* DNA large-M (5 datasets, N = 500..4000, g = 10, k = 6): every row;
* protein (N = 3312, g = 8, k = 4): every row;
* text (N = 6000, g = 8, k = 5): every 23rd row plus the first and last 8
  (the whole matrix would take hours of brute force).

Run from the repository root: ``python tests/golden/make_fullsize_hashes.py``.
It calls only ``oracle`` and the seeded generators in ``synth``; its output,
``tests/golden/fullsize_row_hashes.json``, is what ``test_gpu_fullsize.py``
compares the engine's rows with.
"""

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1704_07468_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "fullsize_row_hashes.json")


def row_digest(K_row, Nm_rows):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(K_row, dtype="<i8").tobytes())
    for r in Nm_rows:
        h.update(np.ascontiguousarray(r, dtype="<i8").tobytes())
    return h.hexdigest()[:16]


def text_rows(n):
    return sorted(set(range(0, n, 23)) | set(range(8)) | set(range(n - 8, n)))


def digests(codes, off, g, k, rows):
    ref = oracle.gram(codes, off, g, k, rows=rows)
    return [row_digest(ref["K"][i], ref["Nm"][:, i]) for i in range(len(rows))]


def main():
    out = {"digest": "sha256(int64 LE K[x,:] then N_0[x,:] .. N_M[x,:])[:16]",
           "datasets": {}}
    jobs = [("dna_toy", 4, 7, 5, synth.dna_toy(), None)]
    for i, ds in enumerate(synth.dna_large()):
        jobs.append((f"dna_large_{i}", 4, 10, 6, ds, None))
    jobs.append(("protein", 20, 8, 4, synth.protein(), None))
    codes, off = synth.text()
    jobs.append(("text", 36, 8, 5, (codes, off), text_rows(len(off) - 1)))
    for name, sigma, g, k, (codes, off), rows in jobs:
        n = len(off) - 1
        rows = list(range(n)) if rows is None else rows
        t0 = time.time()
        hs = digests(codes, off, g, k, np.array(rows, dtype=np.int32))
        out["datasets"][name] = {"sigma": sigma, "g": g, "k": k, "n": n,
                                 "rows": "all" if len(rows) == n else rows,
                                 "digests": hs}
        print(f"{name}: {len(rows)} rows in {time.time() - t0:.1f} s", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main()
