"""Write cube200_trajectory.json: the FP64 oracle's PASD solve of the 200^3 workload.

The workload is the synthetic stand-in for the paper's 200 x 200 x 200
experiments (Section 5): Tucker core 10^3 with Haar factors, 20% of the
entries replaced by U[-1, 1] times max|L0|, R_n = 20, alpha_n = 1/3,
lambda = 1/200, mu0 = 1e-4, rho = 1.1, run until the relative residual
max_n ||T - Z_n - E||_F / ||T||_F falls below 1e-6.

Recorded per iteration: the kept singular value counts s_n (Eq. 13), the
stopping residual and mu. At the end: the iteration count, the Frobenius norms
of L and E, and L, E at seeded sample positions. Only the oracle and the
seeded generator are called; run from the repository root:

    python tests/golden/make_cube200_trajectory.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pasd_oracle as O  # noqa: E402
from paper_1712_09999_gb300 import synth  # noqa: E402

SAMPLE_SEED = 2024
N_SAMPLES = 512


def main():
    pr = synth.cube_200(1)
    T = pr.T.astype(np.float64)
    p = O.Params.from_alpha_lambda((20,) * 3, (1 / 3,) * 3, 1 / 200, stop="fro_rel", tol=1e-6, max_iter=1000)
    res = O.pasd(T, p)
    rng = np.random.default_rng(SAMPLE_SEED)
    idx = np.sort(rng.choice(T.size, size=N_SAMPLES, replace=False))
    Lf, Ef = res.L.reshape(-1), res.E.reshape(-1)
    out = {
        "workload": "200^3, Tucker core 10^3, 20% U[-1,1]*max|L0| corruption, seed 1",
        "ranks": [20, 20, 20], "alpha": [1 / 3] * 3, "lambda": 1 / 200,
        "mu0": p.mu0, "rho": p.rho, "tol": p.tol, "stop": "fro_rel",
        "iters": int(res.iters), "converged": bool(res.converged),
        "kept": [list(map(int, s.kept)) for s in res.trace],
        "res_inf": [float(s.res_inf) for s in res.trace],
        "res_fro_rel": [float(s.res_fro_rel) for s in res.trace],
        "mu_used": [float(s.mu_used) for s in res.trace],
        "L_fro": float(np.linalg.norm(Lf)), "E_fro": float(np.linalg.norm(Ef)),
        "L_max": float(np.abs(Lf).max()), "E_l1": float(np.abs(Ef).sum()),
        "rse": float(O.rse(res.L, pr.L0)),
        "sample_index": idx.tolist(),
        "L_sample": Lf[idx].tolist(), "E_sample": Ef[idx].tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cube200_trajectory.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote %s: %d iterations, converged=%s" % (path, res.iters, res.converged))


if __name__ == "__main__":
    main()
