"""Plain FP64 CPU oracle for PASD, Algorithm 1 of Jiang & Ng,
"Parallel Active Subspace Decomposition for Scalable and Efficient Tensor
Robust Principal Component Analysis" (arXiv 1712.09999).

TEST INFRASTRUCTURE ONLY. This module is the reference the CUDA path is checked
against. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline and ``--impl reference`` arm) may import it; the library never does.
It shares no code with the CUDA path.

Every step follows the paper in the paper's order and notation, with LAPACK
SVDs (numpy.linalg.svd) as the only library primitive besides matrix products:

  Initialise (Algorithm 1): U_n = eye(I_n, R_n), V_n = 0, Y_n = 0, E = 0,
      mu0 = 1e-4, mu_max = 1e10, rho = 1.1.
  U-step (Eq. 9, Eq. 10): orthogonal Procrustes, U = Uhat Vhat^T from the thin
      SVD of G_n V_n^T, with G_n = T_(n) - E_(n) + Y_n,(n) / mu.
  V-step (Eq. 11 - Eq. 13): V_n = SVT_{lambda_n/mu}(U_n^T G_n), SVT as defined
      right after Eq. 13.
  E-step (Eq. 14, Eq. 15): E = prox_{1/(mu N)}(mean_n H_n),
      H_n = T - fold_n(U_n V_n) + Y_n / mu.
  Z_n = fold_n(U_n V_n); Y_n += mu (T - Z_n - E); mu = min(rho mu, mu_max);
  stop when ||T - Z_n - E||_inf < eps for every n (Algorithm 1).
  Output X = sum_n alpha_n Z_n / sum_n alpha_n (Algorithm 1).

Readings where the paper is silent or ambiguous (each is a choice, listed with
its reason in the design notes):
  * Procrustes with a rank-deficient G_n V_n^T (always at k = 0, and whenever
    the SVT zeroes directions): Eq. 10 is then not unique. The oracle keeps the
    unique polar factor on the range of G_n V_n^T and, on the null space of
    V_n^T (the SVT directions with sigma <= tau), takes the isometry closest to
    the previous U_n. At k = 0 this returns eye(I_n, R_n), which is what a thin
    SVD of the zero matrix returns. When every direction is kept it is exactly
    Eq. 10.
  * Weights: lambda_n may be given per mode, or as (alpha_n, lambda) with
    lambda_n = alpha_n / lambda (Theorem 3 writes the objective with alpha_n on
    the nuclear norms and lambda on the l1 norm; dividing by lambda gives Eq. 1).
  * All modes use the iterate of step k (the "parallel" update of Algorithm 1);
    every sub-step of iteration k uses mu^k; mu is raised after the multipliers.
  * The unfolding's column order is C-order over the remaining modes; the
    results do not depend on it (SVT and Procrustes are invariant under a
    common column permutation).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np


# ---------------------------------------------------------------------------
# Tensor basics (Sec. 2.1)
# ---------------------------------------------------------------------------

def unfold(x: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding X_(n) (I_n x prod_{m != n} I_m): the mode-n fibres are the columns."""
    return np.moveaxis(x, n, 0).reshape(x.shape[n], -1)


def fold(m: np.ndarray, n: int, dims: Sequence[int]) -> np.ndarray:
    """fold_n: the tensor A with A_(n) = m (defined after Eq. 3)."""
    dims = tuple(dims)
    rest = dims[:n] + dims[n + 1:]
    return np.moveaxis(m.reshape((dims[n],) + rest), 0, n)


# ---------------------------------------------------------------------------
# Proximal operators
# ---------------------------------------------------------------------------

def soft_threshold(x: np.ndarray, tau: float) -> np.ndarray:
    """prox_tau(x) = sgn(x) max(|x| - tau, 0), elementwise (after Eq. 15)."""
    return np.sign(x) * np.maximum(np.abs(x) - tau, 0.0)


@dataclass
class SvtOut:
    V: np.ndarray        # SVT_tau(X)
    left: np.ndarray     # left singular vectors of X, a full R x R orthogonal basis
    sigma: np.ndarray    # the R singular values of X, descending (zeros past min(R, P))
    kept: int            # number of singular values strictly above tau
    nuclear: float       # ||SVT_tau(X)||_* = sum max(sigma - tau, 0)


def svt(x: np.ndarray, tau: float) -> SvtOut:
    """SVT_tau(X) = U diag(max(Sigma - tau, 0)) V^T from the SVD X = U Sigma V^T
    (definition after Eq. 13). A singular value equal to tau is dropped.

    X is R x P. ``left`` spans all of R^R: when R > P, the R - P directions
    outside the range of X have singular value zero and belong with the other
    dropped directions to the null space of SVT_tau(X)^T."""
    rows, cols = x.shape
    u, s, vt = np.linalg.svd(x, full_matrices=rows > cols)
    if rows > cols:
        vt = vt[:cols]
        s = np.concatenate([s, np.zeros(rows - cols)])
    shrunk = np.maximum(s - tau, 0.0)
    kept = int(np.count_nonzero(s > tau))
    v = (u[:, :kept] * shrunk[:kept]) @ vt[:kept, :]
    return SvtOut(V=v, left=u, sigma=s, kept=kept, nuclear=float(shrunk.sum()))


def procrustes(m: np.ndarray, u_prev: np.ndarray, null_basis: np.ndarray) -> np.ndarray:
    """U-step, Eq. 9 - Eq. 10: argmin_{U in St(I,R)} ||U V - G||_F with M = G V^T.

    ``null_basis`` (R x q, orthonormal columns) spans the null space of V^T, so
    M has rank at most s = R - q. The range part is the polar factor of M on its
    range (Eq. 10 restricted to the s nonzero singular values); the remaining q
    columns are the isometry from the null space into the orthogonal complement
    of that range that is closest to the previous iterate u_prev.
    """
    rows, r = m.shape
    q = null_basis.shape[1]
    s = r - q
    if q:
        m = m - (m @ null_basis) @ null_basis.T
    p1 = np.zeros((rows, r))
    if s:
        uh, sh, vht = np.linalg.svd(m, full_matrices=False)
        if not sh[s - 1] > 0.0:
            raise FloatingPointError("G V^T has rank below the SVT kept count")
        p1 = uh[:, :s] @ vht[:s, :]
    x = np.zeros((rows, r))
    if q:
        b = (u_prev @ null_basis) @ null_basis.T
        b = b - p1 @ (p1.T @ b)
        ub, sb, vbt = np.linalg.svd(b, full_matrices=False)
        if not sb[q - 1] > 0.0:
            raise FloatingPointError("previous subspace degenerate on the null space")
        x = ub[:, :q] @ vbt[:q, :]
    return p1 + x


# ---------------------------------------------------------------------------
# Parameters and state
# ---------------------------------------------------------------------------

def paper_lambdas(dims: Sequence[int]) -> List[float]:
    """lambda_n = sqrt(max(I_n, prod_{m != n} I_m)) / N (Sec. 5.1 setting)."""
    total = int(np.prod(dims))
    n_modes = len(dims)
    return [float(np.sqrt(max(i, total // i))) / n_modes for i in dims]


@dataclass
class Params:
    ranks: Sequence[int]                 # R_n, the rank bounds (1 <= R_n <= I_n)
    lambdas: Sequence[float]             # lambda_n, nuclear weights of Eq. 3
    alpha: Optional[Sequence[float]] = None   # output weights (Algorithm 1 output); None -> equal
    mu0: float = 1e-4
    mu_max: float = 1e10
    rho: float = 1.1
    tol: float = 1e-5
    max_iter: int = 1000
    stop: str = "inf"                    # "inf" (Algorithm 1), "fro_rel", "fixed"

    @staticmethod
    def from_alpha_lambda(ranks, alpha, lam, **kw) -> "Params":
        """(alpha_n, lambda) form of Theorem 3: lambda_n = alpha_n / lambda."""
        return Params(ranks=tuple(ranks), lambdas=tuple(a / lam for a in alpha),
                      alpha=tuple(alpha), **kw)


@dataclass
class State:
    U: List[np.ndarray]
    V: List[np.ndarray]
    null: List[np.ndarray]       # basis of the null space of V_n^T (R_n x q_n)
    E: np.ndarray
    Y: List[np.ndarray]
    mu: float
    k: int = 0


def init_state(T: np.ndarray, ranks: Sequence[int], mu0: float) -> State:
    """Algorithm 1, Initialize: U_n = eye(I_n, R_n), V_n = 0, Y_n = 0, E = 0."""
    dims = T.shape
    total = T.size
    us, vs, nulls, ys = [], [], [], []
    for n, (i_n, r_n) in enumerate(zip(dims, ranks)):
        us.append(np.eye(i_n, r_n))
        vs.append(np.zeros((r_n, total // i_n)))
        nulls.append(np.eye(r_n))        # V = 0: every direction is null
        ys.append(np.zeros(dims))
    return State(U=us, V=vs, null=nulls, E=np.zeros(dims), Y=ys, mu=float(mu0), k=0)


@dataclass
class StepInfo:
    kept: List[int]
    sigma: List[np.ndarray]
    nuclear: List[float]
    A: List[np.ndarray]          # U_n^{k+1 T} G_n^k, the argument of the SVT
    Z: List[np.ndarray]
    res_inf: float               # max_n ||T - Z_n - E||_inf  (Algorithm 1 stop test)
    res_fro_rel: float           # max_n ||T - Z_n - E||_F / ||T||_F
    objective: float             # sum_n lambda_n ||V_n||_* + ||E||_1 (Eq. 3)
    mu_used: float


def step(T: np.ndarray, st: State, p: Params) -> StepInfo:
    """One loop body of Algorithm 1 (modes updated in parallel from iterate k)."""
    dims = T.shape
    n_modes = len(dims)
    mu = st.mu
    new_u, new_v, new_null, zs = [], [], [], []
    kept, sig, nuc, amats = [], [], [], []
    for n in range(n_modes):
        g = unfold(T - st.E + st.Y[n] / mu, n)                  # G_n^k (after Eq. 9)
        m = g @ st.V[n].T                                        # G_n^k V_n^{kT}
        u = procrustes(m, st.U[n], st.null[n])                   # Eq. 10
        a = u.T @ g                                              # argument of Eq. 13
        sv = svt(a, p.lambdas[n] / mu)                           # Eq. 13
        new_u.append(u)
        new_v.append(sv.V)
        new_null.append(sv.left[:, sv.kept:])
        zs.append(fold(u @ sv.V, n, dims))                       # Z_n = fold_n(U_n V_n)
        kept.append(sv.kept)
        sig.append(sv.sigma)
        nuc.append(sv.nuclear)
        amats.append(a)
    h_mean = sum(T - zs[n] + st.Y[n] / mu for n in range(n_modes)) / n_modes   # H_n^k, Eq. 14
    e = soft_threshold(h_mean, 1.0 / (mu * n_modes))             # Eq. 15
    res_inf = 0.0
    res_fro = 0.0
    new_y = []
    for n in range(n_modes):
        r = T - zs[n] - e
        new_y.append(st.Y[n] + mu * r)                           # multiplier update
        res_inf = max(res_inf, float(np.max(np.abs(r))))
        res_fro = max(res_fro, float(np.linalg.norm(r)))
    t_norm = float(np.linalg.norm(T))
    st.U, st.V, st.null, st.E, st.Y = new_u, new_v, new_null, e, new_y
    st.mu = min(p.rho * mu, p.mu_max)                            # mu schedule
    st.k += 1
    obj = sum(l * v for l, v in zip(p.lambdas, nuc)) + float(np.abs(e).sum())
    return StepInfo(kept=kept, sigma=sig, nuclear=nuc, A=amats, Z=zs, res_inf=res_inf,
                    res_fro_rel=res_fro / t_norm if t_norm > 0 else 0.0,
                    objective=obj, mu_used=mu)


def output_low_rank(zs: Sequence[np.ndarray], alpha: Optional[Sequence[float]]) -> np.ndarray:
    """X = sum_n alpha_n Z_n / sum_n alpha_n (Algorithm 1, Output)."""
    if alpha is None:
        alpha = [1.0] * len(zs)
    return sum(a * z for a, z in zip(alpha, zs)) / float(sum(alpha))


@dataclass
class Result:
    L: np.ndarray
    E: np.ndarray
    iters: int
    converged: bool
    trace: List[StepInfo] = field(default_factory=list)
    state: Optional[State] = None


def pasd(T, p: Params, *, keep_trace: bool = True, keep_z_in_trace: bool = False,
         callback=None) -> Result:
    """Algorithm 1 from the initial state until the stop rule holds or max_iter
    loop bodies have run. ``T`` is upcast to float64 first."""
    T = np.asarray(T, dtype=np.float64)
    for n, (i_n, r_n) in enumerate(zip(T.shape, p.ranks)):
        if not 1 <= r_n <= i_n:
            raise ValueError("rank bound must satisfy 1 <= R_n <= I_n")
    st = init_state(T, p.ranks, p.mu0)
    trace: List[StepInfo] = []
    converged = False
    info = None
    while st.k < p.max_iter:
        info = step(T, st, p)
        if callback is not None:
            callback(st, info)
        if keep_trace:
            if not keep_z_in_trace:
                info = StepInfo(**{**info.__dict__, "Z": [], "A": []})
            trace.append(info)
        if p.stop == "inf" and info.res_inf < p.tol:
            converged = True
            break
        if p.stop == "fro_rel" and info.res_fro_rel < p.tol:
            converged = True
            break
    zs = [fold(st.U[n] @ st.V[n], n, T.shape) for n in range(T.ndim)]
    return Result(L=output_low_rank(zs, p.alpha), E=st.E.copy(), iters=st.k,
                  converged=converged, trace=trace, state=st)


def rse(x: np.ndarray, x0: np.ndarray) -> float:
    """Relative square error ||X - T0||_F / ||T0||_F (Sec. 5.1)."""
    return float(np.linalg.norm(x - x0) / np.linalg.norm(x0))
