"""Helpers shared by the parity tests (test code only).

tie_margin: the smallest relative distance min |sigma_i - tau| / tau between a
singular value of the SVT argument A_n and the threshold tau = lambda_n / mu
over every loop body and mode of an oracle trajectory. Identical kept counts on
the GPU and in the oracle say something only if no singular value sat on the
threshold; this margin is that evidence (the SVT keeps sigma > tau strictly).
When PASD_MARGIN_LOG names a file, every margin computed is appended to it as
one JSON line, so a test run leaves the margins of its workloads behind.
"""
import json
import os

import numpy as np


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def tie_margin(trace, lambdas, name=""):
    """min over bodies k, modes n, singular values i of |sigma_i - tau| / tau."""
    best = np.inf
    where = None
    for k, s in enumerate(trace):
        for n, sig in enumerate(s.sigma):
            tau = lambdas[n] / s.mu_used
            m = float(np.min(np.abs(np.asarray(sig) - tau))) / tau
            if m < best:
                best, where = m, (k + 1, n)
    path = os.environ.get("PASD_MARGIN_LOG")
    if path and name:
        with open(path, "a") as f:
            f.write(json.dumps({"workload": name, "tie_margin": best, "body_mode": where}) + "\n")
    return best
