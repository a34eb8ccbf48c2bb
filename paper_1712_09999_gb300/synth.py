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


@dataclass
class RequestSpec:
    """One served solve: a planted tensor with its solver rank bounds."""

    dims: tuple
    tucker: tuple
    rank_bounds: tuple
    rho: float
    seed: int
    kind: str = "planted"    # "planted" (additive) or "hyperspectral" (salt and pepper)


def serving_mix(n: int, seed: int = 4, side_lo: int = 32, side_hi: int = 256) -> list:
    """Request shapes of the serving workload.

    Cube side log-uniform on [side_lo, side_hi]; Tucker rank r_n uniform on
    {3, ..., 20} per mode; rank bound floor(1.2 r_n), at most the side;
    corruption fraction uniform on [0.05, 0.30] (values U[-1,1] max|L0|).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(n):
        side = int(round(float(np.exp(rng.uniform(np.log(side_lo), np.log(side_hi))))))
        tucker = tuple(int(rng.integers(3, 21)) for _ in range(3))
        bounds = tuple(min(side, int(np.floor(1.2 * r))) for r in tucker)
        rho = float(rng.uniform(0.05, 0.30))
        out.append(RequestSpec((side,) * 3, tucker, bounds, rho, 1000 + seed * 100 + q))
    return out


def serving_problem(spec: RequestSpec) -> Problem:
    if spec.kind == "hyperspectral":
        return hyperspectral(spec.dims, spec.tucker, spec.rho, spec.seed)
    return planted(spec.dims, spec.tucker, spec.rho, spec.seed, scale="max", amp=1.0)


def hyperspectral(dims, tucker_ranks, rho: float, seed: int) -> Problem:
    """Hyperspectral-shaped image cube (rows, columns, bands): a Tucker low-rank
    tensor min-max scaled to [0, 1], with exactly floor(rho D) entries (drawn
    without replacement) replaced by 0 or 1 with probability 1/2 each
    (salt-and-pepper noise); E0 = T - L0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = tuple(int(d) for d in dims)
    l0 = tucker_tensor(rng, dims, tucker_ranks)
    lo, hi = float(l0.min()), float(l0.max())
    l0 = (l0 - lo) / (hi - lo) if hi > lo else np.zeros_like(l0)
    total = int(np.prod(dims))
    count = int(np.floor(rho * total))
    support = rng.choice(total, size=count, replace=False) if count else np.zeros(0, np.int64)
    x = l0.reshape(-1).copy()
    x[support] = rng.integers(0, 2, size=count).astype(np.float64)
    x = x.reshape(dims)
    desc = f"hyperspectral tucker{tuple(tucker_ranks)} dims{dims} rho={rho} seed={seed}"
    return Problem(T=x.astype(np.float32), L0=l0, E0=x - l0, support=np.sort(support), desc=desc)


def batch_mix(seed: int = 3, n_random: int = 56, n_hyper: int = 8) -> list:
    """The batched workload: `n_random` planted tensors with every side drawn
    uniformly on {32, ..., 160}, Tucker rank r_n uniform on {3, ..., 15}, additive
    U[-1,1] max|L0| corruption on a fraction uniform on [0.05, 0.30]; plus
    `n_hyper` hyperspectral-shaped 128 x 128 x 191 cubes (spatial ranks uniform on
    {3, ..., 15}, spectral rank 4, salt-and-pepper fraction uniform on [0.05, 0.30]).
    Rank bounds floor(1.2 r_n), at most the side."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(n_random):
        dims = tuple(int(rng.integers(32, 161)) for _ in range(3))
        tucker = tuple(int(rng.integers(3, 16)) for _ in range(3))
        bounds = tuple(min(d, int(np.floor(1.2 * r))) for d, r in zip(dims, tucker))
        out.append(RequestSpec(dims, tucker, bounds, float(rng.uniform(0.05, 0.30)), 3000 + seed * 100 + q))
    for q in range(n_hyper):
        tucker = (int(rng.integers(3, 16)), int(rng.integers(3, 16)), 4)
        dims = (128, 128, 191)
        bounds = tuple(min(d, int(np.floor(1.2 * r))) for d, r in zip(dims, tucker))
        out.append(RequestSpec(dims, tucker, bounds, float(rng.uniform(0.05, 0.30)), 4000 + seed * 100 + q,
                               kind="hyperspectral"))
    return out


def request_precisions(count: int, seed: int = 7) -> np.ndarray:
    """Per-request precision of the serving workload: Bernoulli(1/2), 1 = mixed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, 2, size=count)


def poisson_arrivals(rate: float, count: int, seed: int = 5) -> np.ndarray:
    """Arrival times (seconds from 0) of `count` requests at Poisson rate `rate`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def video(height: int = 144, width: int = 176, frames: int = 300, seed: int = 2,
          n_rect: int = 16, coverage: float = 0.05) -> Problem:
    """Colour-video-shaped tensor, modes (height, width, channel, frame).

    Background: one frame of U[0,1] noise smoothed by a Gaussian of 4 pixels per
    channel and scaled to [0,1], times a per-frame gain 1 + 0.05 U[-1,1], so it is
    rank 1 along the frame mode. Foreground: n_rect rectangles with sides in
    {8, ..., 24}, a random colour in [0,1]^3 and a constant velocity of up to 2
    pixels per frame (reflecting at the borders), each visible over one
    contiguous window of frames sized so that the expected fraction of covered
    voxels is `coverage`. Covered pixels are replaced: E0 = T - L0.
    """
    from scipy.ndimage import gaussian_filter
    rng = np.random.Generator(np.random.PCG64(seed))
    bg = rng.uniform(0.0, 1.0, size=(height, width, 3))
    for c in range(3):
        bg[:, :, c] = gaussian_filter(bg[:, :, c], sigma=4.0, mode="reflect")
    bg = (bg - bg.min()) / max(bg.max() - bg.min(), 1e-12)
    gain = 1.0 + 0.05 * rng.uniform(-1.0, 1.0, size=frames)
    l0 = bg[:, :, :, None] * gain[None, None, None, :]
    t = l0.copy()
    sides = rng.integers(8, 25, size=(n_rect, 2))
    mean_area = float(np.mean(sides[:, 0] * sides[:, 1]))
    always_on = n_rect * mean_area / (height * width)
    win = max(1, min(frames, int(round(frames * coverage / max(always_on, 1e-12)))))
    for q in range(n_rect):
        h, w = int(sides[q, 0]), int(sides[q, 1])
        colour = rng.uniform(0.0, 1.0, size=3)
        y, x = rng.uniform(0, height - h), rng.uniform(0, width - w)
        vy, vx = rng.uniform(-2.0, 2.0), rng.uniform(-2.0, 2.0)
        start = int(rng.integers(0, frames - win + 1))
        for f in range(frames):
            if start <= f < start + win:
                yi, xi = int(y), int(x)
                t[yi:yi + h, xi:xi + w, :, f] = colour
            y += vy
            x += vx
            if y < 0 or y > height - h:
                vy = -vy
                y = min(max(y, 0.0), float(height - h))
            if x < 0 or x > width - w:
                vx = -vx
                x = min(max(x, 0.0), float(width - w))
    e0 = t - l0
    support = np.flatnonzero(e0.reshape(-1) != 0)
    desc = f"video {height}x{width}x3x{frames} rect={n_rect} coverage={coverage} seed={seed}"
    return Problem(T=t.astype(np.float32), L0=l0, E0=e0, support=support, desc=desc)


def planted_device(dims, tucker_ranks, rho: float, seed: int, device, amp: float = 1.0,
                   scale: str = "none"):
    """planted(..., scale=scale) generated on a CUDA device with torch (for sizes and
    counts the host generator is too slow for): Haar factors (QR of a Gaussian matrix,
    columns times sign(diag R)), N(0,1) core, exactly floor(rho D) positions drawn
    without replacement carrying U[-amp, amp] ("none") or U[-amp, amp] max|L0|
    ("max"). Returns (T float32, L0 float32) on `device`; a different random stream
    from planted() for the same seed."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    dims = tuple(int(d) for d in dims)
    core = torch.randn(*tucker_ranks, generator=g, device=device, dtype=torch.float64)
    l0 = core
    for n, (i_n, r_n) in enumerate(zip(dims, tucker_ranks)):
        q, r = torch.linalg.qr(torch.randn(i_n, r_n, generator=g, device=device, dtype=torch.float64))
        q = q * torch.sign(torch.diagonal(r)).unsqueeze(0)
        l0 = torch.movedim(torch.tensordot(q, l0, dims=([1], [n])), 0, n)    # mode-n product
    l0 = l0.to(torch.float32).contiguous()
    total = l0.numel()
    count = int(rho * total)
    t = l0.clone().reshape(-1)
    if scale == "max":
        amp = amp * float(l0.abs().max())
    elif scale != "none":
        raise ValueError(scale)
    if count:
        idx = torch.randperm(total, generator=g, device=device)[:count]
        t[idx] += (torch.rand(count, generator=g, device=device) * 2 - 1) * amp
    return t.reshape(dims), l0
