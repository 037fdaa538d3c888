"""A stand-in chunk estimate for the checkpoint tests that run without a GPU:
the CPU oracle's estimate of small icospheres (vertex rows, 8 walks), a short
sleep per mesh so that a test can interrupt a sweep between meshes."""
import time

import numpy as np

import meshgen
from oracle import oracle as O


def estimate(ids, sleep=0.25):
    out = []
    for i in ids:
        m = meshgen.icosphere(1 + i % 2, radius=1.0 + 0.1 * i)
        rows = O.vertex_rows(m.V, m.F)
        est = O.estimate(m.V, m.F, rows, 8, 1e-3, seed=i, prec=64)
        H = est["H"]
        nnz = (H > 0).sum(1).astype(np.int32)
        bins = [np.flatnonzero(H[v]) for v in range(H.shape[0])]
        out.append(({"hist_bin": np.concatenate(bins).astype(np.int32),
                     "hist_cnt": np.concatenate([H[v, b] for v, b in enumerate(bins)]).astype(np.int32),
                     "hist_nnz": nnz, "omega": O.row_weights(est, rows)},
                    {"stats": {"steps": int(est["steps"].sum())}, "seed": i}))
        time.sleep(sleep)
    return out
