#!/usr/bin/env python3
"""Write the full-size expected values of the build-and-update workload.

The workload: 1e8 3-D points (uniform, or varden-like), BatchInsert of 1e7
new points (ids 1e8 ..), BatchDelete of 1e7 distinct existing ids, default
parameters (lambda 6, phi 32, sample rate 1/64, sigma_os 32, alpha 3/10,
seed 1).  The inputs come from the seeded generators of
paper_2411_09275_gb300/inputs.py, exactly as bench.make_inputs draws them;
every expected value below is computed by the CPU oracle (oracle/) alone:

  export   SHA-256 of the canonical export after the delete (pre-order
           dims uint8, splits int32, sizes uint64, then leaf offsets uint64
           and the sorted leaf ids uint32, all little-endian), and its counts
  knn      SHA-256 of the 10-NN answer (ids uint32, then squared distances
           int64) for 1e4 queries drawn from the same distribution (seed 2)

Run from the repository root (several minutes of one CPU core per case):
    python tests/golden/make_fullsize_golden.py
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2411_09275_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "fullsize_build1e8_d3_ins1e7_del1e7.txt")
N, D, M, K, NQ = 100_000_000, 3, 10_000_000, 10, 10_000


def workload(kind: str):
    X = I.points(kind, N, D, I.SEED_DATA if kind == "uniform" else I.SEED_VARDEN)
    Y = I.points(kind, M, D, I.SEED_INSERT)
    yid = np.arange(N, N + M, dtype=np.uint32)
    zid = I.sample_indices(M, N + M, I.SEED_DELETE).astype(np.uint32)
    Q = I.points(kind, NQ, D, I.SEED_QUERY)
    return X, Y, yid, zid, Q


def export_digest(e: dict) -> str:
    h = hashlib.sha256()
    for key, dt in (("dims", "<u1"), ("splits", "<i4"), ("sizes", "<u8"), ("leaf_offsets", "<u8"),
                    ("leaf_ids", "<u4")):
        h.update(np.ascontiguousarray(e[key], dtype=dt).tobytes())
    return h.hexdigest()


def knn_digest(ids: np.ndarray, d2: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(ids, dtype="<u4").tobytes())
    h.update(np.ascontiguousarray(d2, dtype="<i8").tobytes())
    return h.hexdigest()


def main():
    lines = ["# Expected values of the 1e8-point build + 1e7 insert + 1e7 delete workload (d = 3),",
             "# written by tests/golden/make_fullsize_golden.py from the CPU oracle alone.",
             "# kind key value ..."]
    for kind in ("uniform", "varden"):
        t0 = time.time()
        X, Y, yid, zid, Q = workload(kind)
        t = O.OracleTree(X, None, O.Params(d=D))
        del X
        t.insert(Y, yid)
        nd = t.delete(zid)
        assert nd == M, nd
        e = t.export()
        qi, qd = t.knn(Q, K)
        lines.append(f"{kind} export_sha256 {export_digest(e)}")
        lines.append(f"{kind} nodes {len(e['dims'])} leaves {len(e['leaf_offsets']) - 1} size {t.size} "
                     f"height {t.height}")
        lines.append(f"{kind} knn_sha256 {knn_digest(qi, qd)}")
        lines.append(f"{kind} knn_row0 " + " ".join(f"{int(a)}:{int(b)}" for a, b in zip(qi[0], qd[0])))
        t.close()
        print(kind, f"{time.time() - t0:.0f} s", flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
