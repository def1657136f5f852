"""Writes large_rounding_scalars.json: oracle scalars of two large roundings that the GPU
tests compare against without running the oracle (it needs minutes per train here).

    python tests/golden/make_large_rounding_scalars.py

Calls only the oracle (oracle/core.py, oracle/structured.py) and the shared seeded input
generators.  Cases (both at the full bond ranks of their workloads, with L = 24 sites so that
the unfoldings allow those ranks):

  laplacian3d_r256: x = random TT, L = 24 (3 x 8 bits interleaved), d = 2, rank 256, seed 31,
      cores rounded to FP32; y = 3D Dirichlet Laplacian MPO (rank 7) applied to x (bond
      ranks 1792); z = round(y, 1e-6).
  hadamard_r64: x = random TT, L = 24, d = 2, rank 64, seed 32 (FP64); y = x (.) x (bond
      ranks 4096); z = round(y, 1e-8).  Closed form: the ranks of z are at most
      r (r + 1) / 2 = 2080 (and the unfolding caps).

Stored per case: the ranks of z, ||y||, ||z||, and <z, p_i>, <y, p_i> for three probe
trains p_i = random TT (L = 24, d = 2, rank 3, seeds 900..902).  The rounding is the
oracle's (Section 3.2: right-to-left orthogonalisation, then truncated SVDs at
eps ||y|| / sqrt(L - 1) per bond); inner products and norms are exact sums (Section 3.1).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import core, structured  # noqa: E402
from paper_2602_20226_gb300 import inputs  # noqa: E402

L = 24
PROBES = [inputs.random_tt(900 + i, L, 2, 3) for i in range(3)]


def case_laplacian3d():
    x = [c.astype(np.float32).astype(np.float64) for c in inputs.random_tt(31, L, 2, 256)]
    w = structured.laplacian_mpo(3, L // 3)
    y = core.apply_mpo(w, x)
    return y, 1e-6


def case_hadamard():
    x = inputs.random_tt(32, L, 2, 64)
    return core.hadamard(x, x), 1e-8


def scalars(y, eps):
    t0 = time.time()
    z = core.round_tt(y, eps)
    return {
        "eps": eps,
        "ranks_y": core.ranks(y),
        "ranks_z": core.ranks(z),
        "norm_y": core.norm(y),
        "norm_z": core.norm(z),
        "inner_z_p": [core.inner(z, p) for p in PROBES],
        "inner_y_p": [core.inner(y, p) for p in PROBES],
        "oracle_seconds": round(time.time() - t0, 1),
    }


def main():
    out = {"L": L, "probes": "random_tt(900 + i, 24, 2, 3), i = 0, 1, 2"}
    for name, make in (("laplacian3d_r256", case_laplacian3d), ("hadamard_r64", case_hadamard)):
        y, eps = make()
        out[name] = scalars(y, eps)
        print(name, out[name]["ranks_z"], out[name]["oracle_seconds"], "s", flush=True)
        del y
    with open(os.path.join(HERE, "large_rounding_scalars.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
