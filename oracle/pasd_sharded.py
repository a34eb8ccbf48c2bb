"""Slab-sharded form of the oracle's loop body (Algorithm 1) over several ranks.

TEST INFRASTRUCTURE ONLY, like ``pasd_oracle``: the plan it checks is how one
solve would be split over several GPUs, each holding one slab of the tensor.
Only ``tests/`` use it. Plain FP64 NumPy; it shares no code with the CUDA path.

The tensor is cut along one mode m into contiguous slabs of the index i_m, one
per rank (a rank may hold none). T, E and Y_n live slab by slab. Every step of
Algorithm 1 is then local to a slab or needs one of these exchanges:

  mode n != m: the columns of G_(n), A_n and V_n are split with the slabs, the
    rows are not. G_n V_n^T (the argument of Eq. 10) is a sum over columns:
    an all-reduce of I_n x R_n. The SVT of A_n (Eq. 13) needs the singular
    values and left singular vectors of a column-split R_n-row matrix: an
    all-gather of one R_n x R_n triangular factor per rank (below). U_n is the
    same on every rank.
  mode m: the rows of G_(m), U_m and G_m V_m^T are split, the columns are not.
    The polar factor of Eq. 10 needs the right singular vectors of row-split
    R_m-column matrices: one or two all-gathers of R_m x R_m triangular
    factors and, with a null space, one all-reduce of R_m x R_m.
    A_m = U_m^T G_m sums over rows: an all-reduce of R_m x P_m (a
    reduce-scatter followed by an all-gather). V_m is the same on every rank.
  E-step (Eq. 14, Eq. 15), multipliers and Z_n are elementwise on the slab.
  Stop test: an all-reduce (max) of ||T - Z_n - E||_inf and an all-reduce
    (sum) of the N squared Frobenius norms and ||E||_1 (and, once before the
    first body, of ||T||_F^2 for the relative residual).

The small factors come from a tall-skinny QR: each rank factors its own rows
(X_r = Q_r R_r), the R_r are gathered and the stack is factored again, which
gives the R factor of the whole X; X and that R factor share their singular
values and right singular vectors. An R x R SVD of it then gives SVT_tau(A) =
W diag(max(1 - tau/sigma, 0)) W^T A (W, sigma from A^T = Q R) and the polar
factor of X on its s-dimensional range, X W_s diag(1/sigma_s) W_s^T. Gram
matrices (X^T X, A A^T) would carry the same information in one all-reduce,
but square the condition number: directions the SVT has just kept have
singular values barely above zero in G_n V_n^T, and there the Gram route loses
them in FP64. ``pasd_oracle`` takes both from LAPACK SVDs of the whole matrices,
so agreement between the two checks the exchange plan and this route. The
readings are those of ``pasd_oracle`` (the null-space rule of the U-step,
parallel modes, mu^k in every sub-step).
"""
from __future__ import annotations

from collections import Counter
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

from .pasd_oracle import Params, soft_threshold


# ---------------------------------------------------------------------------
# Collectives
# ---------------------------------------------------------------------------

class Comm:
    """The three collectives the sharded body needs, on one rank of ``world``.

    The base class is a single rank (every collective is the identity).
    ``elements`` counts the values this rank contributed to each kind of exchange."""

    def __init__(self, rank: int = 0, world: int = 1):
        self.rank = rank
        self.world = world
        self.elements: Counter = Counter()

    def _sum(self, x: np.ndarray) -> np.ndarray:
        return x

    def _max(self, x: float) -> float:
        return x

    def _gather(self, x: np.ndarray) -> np.ndarray:
        return x

    def sum(self, x: np.ndarray, kind: str) -> np.ndarray:
        """Elementwise sum of x over all ranks (every rank gets the same result)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        self.elements[kind] += x.size
        return self._sum(x)

    def max(self, x: float, kind: str) -> float:
        self.elements[kind] += 1
        return float(self._max(float(x)))

    def gather(self, x: np.ndarray, kind: str) -> np.ndarray:
        """Every rank's x stacked along the first axis in rank order (same on every rank)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        self.elements[kind] += x.size
        return self._gather(x)


class DistComm(Comm):
    """Collectives over an initialised ``torch.distributed`` process group (CPU tensors)."""

    def __init__(self, dist):
        super().__init__(dist.get_rank(), dist.get_world_size())
        self._dist = dist

    def _sum(self, x):
        import torch
        t = torch.from_numpy(x.copy())
        self._dist.all_reduce(t, op=self._dist.ReduceOp.SUM)
        return t.numpy()

    def _max(self, x):
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self._dist.all_reduce(t, op=self._dist.ReduceOp.MAX)
        return float(t.item())

    def _gather(self, x):
        import torch
        t = torch.from_numpy(x.copy())
        parts = [torch.empty_like(t) for _ in range(self.world)]
        self._dist.all_gather(parts, t)
        return torch.cat(parts, 0).numpy()


def slab_bounds(length: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous ranges [lo, hi) of i_m per rank; the first length % world ranks get one more."""
    base, extra = divmod(length, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


# ---------------------------------------------------------------------------
# Local pieces
# ---------------------------------------------------------------------------

def _unfold(x: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding of a (possibly empty) slab: the mode-n fibres are the columns."""
    cols = int(np.prod([d for i, d in enumerate(x.shape) if i != n]))
    return np.moveaxis(x, n, 0).reshape(x.shape[n], cols)


def _fold(m: np.ndarray, n: int, dims: Sequence[int]) -> np.ndarray:
    dims = tuple(dims)
    return np.moveaxis(m.reshape((dims[n],) + dims[:n] + dims[n + 1:]), 0, n)


def _tall_r(x_loc: np.ndarray, gather) -> np.ndarray:
    """R factor (R x R) of a tall matrix X whose rows may be split across ranks: each
    rank's own R factor, zero-padded to R x R, is stacked by ``gather`` and factored
    again (tall-skinny QR). X^T X = R^T R."""
    r = x_loc.shape[1]
    own = np.zeros((r, r))
    if x_loc.shape[0]:
        f = np.linalg.qr(x_loc, mode="r")
        own[:f.shape[0]] = f
    return np.linalg.qr(gather(own), mode="r")


def _range_polar(x_loc: np.ndarray, s: int, gather) -> np.ndarray:
    """Polar factor of X on the span of its s largest singular directions (Eq. 10),
    X W_s diag(1/sigma_s) W_s^T, for X whose rows may be split across ranks."""
    _, sig, wt = np.linalg.svd(_tall_r(x_loc, gather))
    if not sig[s - 1] > 0.0:
        raise FloatingPointError("polar factor: matrix has rank below the kept count")
    ws = wt[:s].T
    return x_loc @ (ws / sig[:s]) @ ws.T


def _procrustes(m_loc: np.ndarray, u_prev_loc: np.ndarray, null: np.ndarray, gather, total) -> np.ndarray:
    """U-step (Eq. 9, Eq. 10) with the oracle's null-space reading, rows possibly split
    (``gather`` stacks R x R blocks over the ranks, ``total`` sums R x R over them).

    The polar factor of M on its range (M restricted to the kept directions), plus, on
    the null space of V^T (columns of ``null``), the isometry into the complement of
    that range closest to the previous iterate."""
    r = m_loc.shape[1]
    q = null.shape[1]
    s = r - q
    if q:
        m_loc = m_loc - (m_loc @ null) @ null.T
    p1 = _range_polar(m_loc, s, gather) if s else np.zeros_like(m_loc)
    x = np.zeros_like(m_loc)
    if q:
        b = (u_prev_loc @ null) @ null.T
        if s:
            b = b - p1 @ total(p1.T @ b)
        x = _range_polar(b, q, gather)
    return p1 + x


def _svt(a_loc: np.ndarray, tau: float, gather):
    """SVT_tau(A) (definition after Eq. 13) for a short-fat A whose columns may be split
    across ranks: W and sigma from the SVD of the R factor of A^T, then
    W diag(max(1 - tau/sigma, 0)) W^T A on each rank's columns. A singular value
    equal to tau is dropped."""
    _, sigma, wt = np.linalg.svd(_tall_r(a_loc.T, gather))
    w = wt.T
    kept = int(np.count_nonzero(sigma > tau))
    wk = w[:, :kept]
    v_loc = (wk * (1.0 - tau / sigma[:kept])) @ (wk.T @ a_loc)
    nuclear = float(np.maximum(sigma - tau, 0.0).sum())
    return v_loc, np.ascontiguousarray(w[:, kept:]), sigma, kept, nuclear


# ---------------------------------------------------------------------------
# Sharded state and loop body
# ---------------------------------------------------------------------------

@dataclass
class ShardState:
    U: List[np.ndarray]      # n != m: I_n x R_n (same on every rank); n == m: slab rows x R_m
    V: List[np.ndarray]      # n != m: R_n x slab columns; n == m: R_m x P_m (same on every rank)
    null: List[np.ndarray]   # R_n x q_n basis of the null space of V_n^T (same on every rank)
    E: np.ndarray            # slab of E
    Y: List[np.ndarray]      # slabs of Y_n
    mu: float
    k: int = 0


@dataclass
class ShardStep:
    kept: List[int]
    res_inf: float
    res_fro_rel: float
    objective: float
    mu_used: float


def init_shard(dims: Sequence[int], ranks: Sequence[int], m: int, lo: int, hi: int,
               mu0: float) -> ShardState:
    """Algorithm 1, Initialize, restricted to the slab lo <= i_m < hi."""
    local = list(dims)
    local[m] = hi - lo
    size = int(np.prod(local))
    us, vs, nulls, ys = [], [], [], []
    for n, (i_n, r_n) in enumerate(zip(dims, ranks)):
        eye = np.eye(i_n, r_n)
        if n == m:
            us.append(eye[lo:hi].copy())
            vs.append(np.zeros((r_n, int(np.prod(dims)) // i_n)))
        else:
            us.append(eye)
            vs.append(np.zeros((r_n, size // i_n)))
        nulls.append(np.eye(r_n))
        ys.append(np.zeros(local))
    return ShardState(U=us, V=vs, null=nulls, E=np.zeros(local), Y=ys, mu=float(mu0))


def shard_step(T_loc: np.ndarray, st: ShardState, p: Params, m: int, t_norm: float,
               comm: Comm) -> ShardStep:
    """One loop body of Algorithm 1 on this rank's slab (all modes from iterate k)."""
    n_modes = T_loc.ndim
    mu = st.mu
    local = T_loc.shape

    def gather(kind):
        return lambda x: comm.gather(x, kind)

    def total(kind):
        return lambda x: comm.sum(x, kind)

    def here(x):
        return x

    new_u, new_v, new_null, zs, kept, nuc = [], [], [], [], [], []
    for n in range(n_modes):
        g = _unfold(T_loc - st.E + st.Y[n] / mu, n)                 # this rank's part of G_n^k
        tau = p.lambdas[n] / mu
        if n != m:
            mm = comm.sum(g @ st.V[n].T, "M")                        # G_n^k V_n^{kT}, Eq. 10
            u = _procrustes(mm, st.U[n], st.null[n], here, here)
            v, null, _, s, nn = _svt(u.T @ g, tau, gather("rfac"))  # Eq. 13
        else:
            u = _procrustes(g @ st.V[n].T, st.U[n], st.null[n], gather("rfac"), total("proj"))
            a = comm.sum(u.T @ g, "A")                               # U_m^T G_m, summed over rows
            v, null, _, s, nn = _svt(a, tau, here)
        new_u.append(u)
        new_v.append(v)
        new_null.append(null)
        zs.append(_fold(u @ v, n, local))                            # slab of Z_n
        kept.append(s)
        nuc.append(nn)
    h_mean = sum(T_loc - zs[n] + st.Y[n] / mu for n in range(n_modes)) / n_modes   # Eq. 14
    e = soft_threshold(h_mean, 1.0 / (mu * n_modes))                 # Eq. 15
    r_inf = 0.0
    sums = np.zeros(n_modes + 1)
    new_y = []
    for n in range(n_modes):
        r = T_loc - zs[n] - e
        new_y.append(st.Y[n] + mu * r)
        r_inf = max(r_inf, float(np.max(np.abs(r), initial=0.0)))
        sums[n] = float(np.sum(r * r))
    sums[n_modes] = float(np.abs(e).sum())
    r_inf = comm.max(r_inf, "stop")
    sums = comm.sum(sums, "stop")
    st.U, st.V, st.null, st.E, st.Y = new_u, new_v, new_null, e, new_y
    st.mu = min(p.rho * mu, p.mu_max)
    st.k += 1
    fro = float(np.sqrt(np.max(sums[:n_modes])))
    obj = sum(l * v for l, v in zip(p.lambdas, nuc)) + float(sums[n_modes])
    return ShardStep(kept=kept, res_inf=r_inf, res_fro_rel=fro / t_norm if t_norm > 0 else 0.0,
                     objective=obj, mu_used=mu)


@dataclass
class ShardResult:
    L: np.ndarray            # slab of the output low-rank tensor
    E: np.ndarray            # slab of E
    iters: int
    converged: bool
    trace: List[ShardStep] = field(default_factory=list)
    state: Optional[ShardState] = None


def pasd_sharded(T_loc, dims: Sequence[int], m: int, lo: int, hi: int, p: Params,
                 comm: Comm) -> ShardResult:
    """Algorithm 1 on the slab lo <= i_m < hi of a tensor of shape ``dims``; every rank
    of ``comm`` calls this with its own slab, and the slabs tile the mode-m range."""
    T_loc = np.asarray(T_loc, dtype=np.float64)
    dims = tuple(int(d) for d in dims)
    expect = list(dims)
    expect[m] = hi - lo
    if T_loc.shape != tuple(expect):
        raise ValueError("slab shape does not match dims and [lo, hi)")
    for i_n, r_n in zip(dims, p.ranks):
        if not 1 <= r_n <= i_n:
            raise ValueError("rank bound must satisfy 1 <= R_n <= I_n")
    t_norm = float(np.sqrt(comm.sum(np.array([np.sum(T_loc * T_loc)]), "init")[0]))
    st = init_shard(dims, p.ranks, m, lo, hi, p.mu0)
    trace: List[ShardStep] = []
    converged = False
    while st.k < p.max_iter:
        info = shard_step(T_loc, st, p, m, t_norm, comm)
        trace.append(info)
        if p.stop == "inf" and info.res_inf < p.tol:
            converged = True
            break
        if p.stop == "fro_rel" and info.res_fro_rel < p.tol:
            converged = True
            break
    local = T_loc.shape
    zs = [_fold(st.U[n] @ st.V[n], n, local) for n in range(T_loc.ndim)]
    alpha = p.alpha if p.alpha is not None else [1.0] * len(zs)
    L = sum(a * z for a, z in zip(alpha, zs)) / float(sum(alpha))
    return ShardResult(L=L, E=st.E.copy(), iters=st.k, converged=converged, trace=trace, state=st)


def exchange_elements(dims: Sequence[int], ranks: Sequence[int], m: int, kept_before: Sequence[int]) -> dict:
    """Values one rank contributes to each kind of exchange in one loop body of the
    sharded plan, given the kept counts of the previous body (0 before the first)."""
    n_modes = len(dims)
    total = int(np.prod(dims))
    out = Counter()
    for n in range(n_modes):
        r = ranks[n]
        if n != m:
            out["M"] += dims[n] * r
            out["rfac"] += r * r
        else:
            s = kept_before[n]
            q = r - s
            out["rfac"] += r * r * ((1 if s else 0) + (1 if q else 0))
            if s and q:
                out["proj"] += r * r
            out["A"] += r * (total // dims[n])
    out["stop"] += 1 + n_modes + 1
    return dict(out)
