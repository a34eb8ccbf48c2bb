"""Seeded synthetic inputs for tensor robust PCA (planted low-rank + sparse).

This module generates inputs only; it holds none of the solver's arithmetic, so
both the CUDA path and the FP64 oracle may use it.

Workload families (Sec. 5.1 of the paper, "Synthetic Tensor Recovery"):
  * the ground truth T0 is a Tucker tensor: a core with N(0, 1) entries multiplied
    along each mode by a column-orthonormal factor drawn from the Haar measure;
  * a random fraction rho of the entries is corrupted additively.
The paper draws the corruption from U[-1, 1]; the larger workloads scale it (by
std(T0) or max|T0|) so that the outliers dominate the low-rank signal.

Every generator takes an explicit integer seed and uses numpy's PCG64.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def haar_orthonormal(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """Column-orthonormal rows x cols matrix from the Haar measure.

    QR of a Gaussian matrix with the columns of Q multiplied by sign(diag(R)),
    which makes the distribution exactly Haar (Mezzadri, 2007).
    """
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


def tucker_tensor(rng: np.random.Generator, dims, ranks) -> np.ndarray:
    """Core with N(0,1) entries times Haar factors along every mode (FP64)."""
    core = rng.standard_normal(tuple(ranks))
    x = core
    for n, (i_n, r_n) in enumerate(zip(dims, ranks)):
        u = haar_orthonormal(rng, i_n, r_n)
        x = np.moveaxis(np.tensordot(u, np.moveaxis(x, n, 0), axes=(1, 0)), 0, n)
    return np.ascontiguousarray(x)


@dataclass
class Problem:
    """A planted problem: T = L0 + E0 (float32 observation) and its FP64 truth."""

    T: np.ndarray        # float32, C-order, the observed tensor
    L0: np.ndarray       # float64 ground-truth low-rank part
    E0: np.ndarray       # float64 ground-truth sparse part (T = L0 + E0 before rounding)
    support: np.ndarray  # flat indices of the corrupted entries
    desc: str


def planted(dims, tucker_ranks, rho: float, seed: int, *, scale: str = "none",
            amp: float = 1.0) -> Problem:
    """Tucker low-rank tensor plus sparse additive corruption.

    ``rho``   fraction of corrupted entries; exactly floor(rho * D) positions are
              drawn uniformly without replacement.
    ``scale`` "none": values U[-amp, amp] (the paper's Table 1 setting, amp=1);
              "std":  U[-amp, amp] * std(L0);
              "max":  U[-amp, amp] * max|L0|.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = tuple(int(d) for d in dims)
    l0 = tucker_tensor(rng, dims, tucker_ranks)
    total = int(np.prod(dims))
    count = int(np.floor(rho * total))
    support = rng.choice(total, size=count, replace=False) if count else np.zeros(0, np.int64)
    vals = rng.uniform(-amp, amp, size=count)
    if scale == "std":
        vals = vals * float(np.std(l0))
    elif scale == "max":
        vals = vals * float(np.max(np.abs(l0)))
    elif scale != "none":
        raise ValueError(scale)
    e0 = np.zeros(total)
    e0[support] = vals
    e0 = e0.reshape(dims)
    t = (l0 + e0).astype(np.float32)
    desc = f"tucker{tuple(tucker_ranks)} dims{dims} rho={rho} scale={scale} amp={amp} seed={seed}"
    return Problem(T=t, L0=l0, E0=e0, support=np.sort(support), desc=desc)


def cube_small(seed: int = 0) -> Problem:
    """50x50x50, Tucker core 5^3, 10% corruption U[-10,10]*std(L0)."""
    return planted((50, 50, 50), (5, 5, 5), 0.10, seed, scale="std", amp=10.0)


def cube_200(seed: int = 1) -> Problem:
    """200x200x200, Tucker core 10^3, 20% corruption U[-1,1]*max|L0|."""
    return planted((200, 200, 200), (10, 10, 10), 0.20, seed, scale="max", amp=1.0)


def table1(dims, rho: float, seed: int, r: int = 10) -> Problem:
    """The paper's Table 1 family: Tucker rank r per mode, U[-1,1] additive noise."""
    return planted(dims, (r,) * len(dims), rho, seed, scale="none", amp=1.0)


def random_tensor(dims, seed: int, dtype=np.float32) -> np.ndarray:
    """Unstructured N(0,1) tensor (kernel-level tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(tuple(dims)).astype(dtype)
