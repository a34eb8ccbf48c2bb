"""Pins for the FP64 oracle: each test checks it against something the paper or
the mathematics fixes, not against its own formulas retyped."""
import numpy as np
import pytest

from oracle import pasd_oracle as O
from paper_1712_09999_gb300 import synth


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# --- proximal operators ----------------------------------------------------

def test_soft_threshold_is_the_l1_prox_by_brute_force():
    # prox_tau(x) = argmin_e tau|e| + (e - x)^2 / 2 (after Eq. 15), checked on a grid.
    rng = _rng(1)
    grid = np.linspace(-6, 6, 240001)
    for _ in range(40):
        x = rng.uniform(-5, 5)
        tau = rng.uniform(0, 3)
        f = tau * np.abs(grid) + 0.5 * (grid - x) ** 2
        e_star = grid[np.argmin(f)]
        assert abs(O.soft_threshold(np.array(x), tau) - e_star) < 1e-4


def test_e_step_minimises_eq14_elementwise():
    # Eq. 14 is separable: min_e |e| + mu/2 sum_n (e - h_n)^2; Eq. 15 claims the
    # minimiser is prox_{1/(mu N)}(mean h). Brute force on a grid.
    rng = _rng(2)
    grid = np.linspace(-8, 8, 320001)
    for n_modes in (2, 3, 4):
        for _ in range(15):
            h = rng.uniform(-4, 4, size=n_modes)
            mu = rng.uniform(0.2, 5)
            f = np.abs(grid) + 0.5 * mu * ((grid[:, None] - h[None, :]) ** 2).sum(1)
            e_star = grid[np.argmin(f)]
            e = O.soft_threshold(np.array(h.mean()), 1.0 / (mu * n_modes))
            assert abs(e - e_star) < 1e-4


def test_svt_closed_form_on_constructed_matrices():
    # X = Q1 diag(s) Q2^T with known orthonormal factors: SVT_tau(X) = Q1 diag((s-tau)+) Q2^T.
    rng = _rng(3)
    for (r, p) in ((3, 7), (4, 4), (5, 2), (1, 6)):
        k = min(r, p)
        q1 = synth.haar_orthonormal(rng, r, k)
        q2 = synth.haar_orthonormal(rng, p, k)
        s = np.sort(rng.uniform(0.1, 5, size=k))[::-1]
        tau = float(0.5 * (s[k // 2] + s[k // 2 - 1])) if k > 1 else float(0.5 * s[0])
        x = (q1 * s) @ q2.T
        out = O.svt(x, tau)
        want = (q1 * np.maximum(s - tau, 0)) @ q2.T
        assert np.allclose(out.V, want, atol=1e-12)
        assert out.kept == int(np.sum(s > tau))
        assert out.nuclear == pytest.approx(np.maximum(s - tau, 0).sum(), abs=1e-12)


def test_svt_drops_a_singular_value_equal_to_tau():
    # SVT_tau keeps max(sigma - tau, 0): a singular value exactly at tau contributes
    # nothing and is not counted as kept (the tie reading of the SVT definition).
    # Signed permutations of a diagonal have exact singular values 3, 2, 0.5.
    rng = _rng(31)
    for _ in range(6):
        perm = rng.permutation(5)
        x = np.zeros((3, 5))
        x[np.arange(3), perm[:3]] = np.array([3.0, 2.0, 0.5]) * rng.choice([-1.0, 1.0], 3)
        out = O.svt(x, 2.0)
        assert out.kept == 1
        assert out.nuclear == 1.0
        assert np.allclose(out.V, np.where(np.abs(x) == 3.0, np.sign(x), 0.0), atol=1e-15)


def test_svt_is_the_nuclear_prox():
    # SVT_tau(X) minimises tau ||V||_* + ||V - X||_F^2 / 2 (strongly convex), so no
    # perturbation can lower the objective.
    rng = _rng(4)
    for _ in range(10):
        x = rng.standard_normal((4, 9))
        tau = float(np.linalg.svd(x, compute_uv=False)[1])
        v = O.svt(x, tau).V
        f = lambda m: tau * np.linalg.svd(m, compute_uv=False).sum() + 0.5 * np.sum((m - x) ** 2)
        f0 = f(v)
        for _ in range(200):
            d = rng.standard_normal(x.shape) * rng.choice([1e-1, 1e-3])
            assert f(v + d) >= f0 - 1e-12


def test_svt_orthogonal_left_invariance():
    # SVT_tau(Q J) = Q SVT_tau(J) for Q^T Q = I: the step from Eq. 11 to Eq. 12.
    rng = _rng(5)
    for (i, r, p) in ((9, 4, 11), (6, 6, 3), (20, 3, 30)):
        q = synth.haar_orthonormal(rng, i, r)
        j = rng.standard_normal((r, p))
        tau = 0.7
        assert np.allclose(O.svt(q @ j, tau).V, q @ O.svt(j, tau).V, atol=1e-12)


# --- Procrustes (Eq. 9, Eq. 10) -------------------------------------------

def _stiefel_samples(rng, i, r, count):
    g = rng.standard_normal((count, i, r))
    q, rr = np.linalg.qr(g)
    return q


def test_procrustes_full_rank_is_the_global_minimiser():
    rng = _rng(6)
    for (i, r, p) in ((3, 2, 5), (4, 2, 6), (4, 3, 8)):
        v = rng.standard_normal((r, p))
        g = rng.standard_normal((i, p))
        u = O.procrustes(g @ v.T, np.eye(i, r), np.zeros((r, 0)))
        assert np.allclose(u.T @ u, np.eye(r), atol=1e-12)
        f = lambda uu: np.sum((uu @ v - g) ** 2, axis=(-2, -1))
        samples = _stiefel_samples(rng, i, r, 200000)
        assert f(u) <= f(samples).min() + 1e-12
        # local optimality along the manifold: U exp(S) for skew S, plus the
        # complement directions via a full orthogonal rotation from the left
        for _ in range(100):
            a = rng.standard_normal((i, i)) * 1e-3
            rot = np.linalg.qr(np.eye(i) + (a - a.T))[0]
            rot = rot * np.sign(np.diag(np.linalg.qr(np.eye(i) + (a - a.T))[1]))
            assert f(rot @ u) >= f(u) - 1e-12


def test_procrustes_rank_deficient_is_a_minimiser_and_closest_on_null_space():
    rng = _rng(7)
    i, r, p = 5, 3, 9
    # V with one zero row in a rotated basis: rank(V) = 2, null space of V^T is 1-D
    w = synth.haar_orthonormal(rng, r, r)
    core = rng.standard_normal((r, p))
    core[2] = 0.0
    v = w @ core
    null = w[:, 2:]
    g = rng.standard_normal((i, p))
    u_prev = synth.haar_orthonormal(rng, i, r)
    u = O.procrustes(g @ v.T, u_prev, null)
    assert np.allclose(u.T @ u, np.eye(r), atol=1e-12)
    f = lambda uu: np.sum((uu @ v - g) ** 2, axis=(-2, -1))
    samples = _stiefel_samples(rng, i, r, 200000)
    assert f(u) <= f(samples).min() + 1e-12
    # among the minimisers (free on the null direction), U is closest to u_prev there:
    # any other unit vector orthogonal to range(U w_kept) is no closer to u_prev @ null.
    x = u @ null
    target = u_prev @ null
    comp = np.eye(i) - (u @ w[:, :2]) @ (u @ w[:, :2]).T
    for _ in range(2000):
        y = comp @ rng.standard_normal((i, 1))
        y /= np.linalg.norm(y)
        assert np.sum((x - target) ** 2) <= np.sum((y - target) ** 2) + 1e-12
    # basis-free: another orthonormal basis of the same null space gives the same U
    assert np.allclose(O.procrustes(g @ v.T, u_prev, -null), u, atol=1e-12)


def test_procrustes_at_initialisation_keeps_eye():
    # Algorithm 1 starts from V = 0: G V^T = 0 and a thin SVD of the zero matrix returns
    # eye(I, R) as its left factor and eye(R) as its right factor.
    for (i, r) in ((5, 2), (7, 7), (4, 1)):
        u = O.procrustes(np.zeros((i, r)), np.eye(i, r), np.eye(r))
        assert np.array_equal(u, np.eye(i, r))


# --- Algorithm 1 as a whole -----------------------------------------------

def _small_problem(seed=11, dims=(12, 10, 8), ranks=(2, 2, 2), rho=0.1):
    return synth.planted(dims, ranks, rho, seed, scale="std", amp=5.0)


def test_idle_phase_matches_closed_form():
    # While V_n = 0 and E = 0, Algorithm 1 reduces to Y^k = mu0 T (rho^k - 1)/(rho - 1),
    # U = eye, and the first activation happens at the first k with
    #   sigma_max(first R rows of c_k T_(n)) > lambda_n / mu^k   (SVT of Eq. 13), or
    #   c_k max|T| > 1/(mu^k N)                                    (prox of Eq. 15),
    # where c_k = 1 + (1 - rho^-k)/(rho - 1) so that G^k = c_k T.
    pr = _small_problem()
    t = pr.T.astype(np.float64)
    dims = t.shape
    n_modes = len(dims)
    ranks = (3, 3, 3)
    lam = O.paper_lambdas(dims)
    p = O.Params(ranks=ranks, lambdas=lam, stop="fixed", max_iter=400)
    mu0, rho = p.mu0, p.rho
    k_pred = None
    for k in range(400):
        mu = mu0 * rho ** k
        c = 1.0 + (1.0 - rho ** (-k)) / (rho - 1.0)
        svt_on = any(np.linalg.svd(c * O.unfold(t, n)[:ranks[n]], compute_uv=False)[0] > lam[n] / mu
                     for n in range(n_modes))
        e_on = c * np.max(np.abs(t)) > 1.0 / (mu * n_modes)
        if svt_on or e_on:
            k_pred = k
            break
    assert k_pred is not None and k_pred > 5
    st = O.init_state(t, ranks, p.mu0)
    for k in range(k_pred + 1):
        y_closed = mu0 * t * (rho ** k - 1.0) / (rho - 1.0)
        for n in range(n_modes):
            assert np.allclose(st.Y[n], y_closed, rtol=1e-12, atol=1e-300)
            assert np.allclose(st.U[n], np.eye(dims[n], ranks[n]), rtol=0, atol=1e-12)
            assert not np.any(st.V[n])
        assert not np.any(st.E)
        info = O.step(t, st, p)
        if k < k_pred:
            assert max(info.kept) == 0 and not np.any(st.E)
    assert max(info.kept) > 0 or np.any(st.E)


def test_multiplier_sum_bound_eqS1():
    # First-order optimality of the E-step gives ||sum_n Y_n^{k+1}||_inf <= 1 (App. A).
    pr = _small_problem(seed=12)
    t = pr.T.astype(np.float64)
    p = O.Params(ranks=(3, 3, 3), lambdas=O.paper_lambdas(t.shape), stop="fixed", max_iter=260)
    st = O.init_state(t, p.ranks, p.mu0)
    hit_one = False
    for _ in range(p.max_iter):
        info = O.step(t, st, p)
        s = np.max(np.abs(sum(st.Y)))
        # Y_n accumulates mu * (T - Z_n - E): its rounding error scales with eps * mu * |T|
        slack = 1e-12 + 64 * np.finfo(float).eps * info.mu_used * np.abs(t).max()
        assert s <= 1.0 + slack
        hit_one |= s > 1.0 - slack
    assert hit_one   # E became nonzero, so the bound is attained on its support


def test_dual_spectral_bound_eqS3():
    # ||U_n^T Yhat_n,(n)||_2 <= lambda_n with Yhat from Eq. 16 (App. A).
    pr = _small_problem(seed=13)
    t = pr.T.astype(np.float64)
    p = O.Params(ranks=(3, 3, 3), lambdas=O.paper_lambdas(t.shape), stop="fixed", max_iter=240)
    st = O.init_state(t, p.ranks, p.mu0)
    active = 0
    for _ in range(p.max_iter):
        y_old = [y.copy() for y in st.Y]
        e_old = st.E.copy()
        info = O.step(t, st, p)
        for n in range(3):
            yhat = y_old[n] + info.mu_used * (t - info.Z[n] - e_old)
            nrm = np.linalg.norm(st.U[n].T @ O.unfold(yhat, n), 2)
            assert nrm <= p.lambdas[n] * (1 + 1e-9)
            active += info.kept[n] > 0
    assert active > 0


def _horpca(t, lambdas, iters, mu0=1e-4, rho=1.1, mu_max=1e10):
    # Independent HoRPCA ADMM for Eq. 2 (Goldfarb & Qin): Z_n = SVT of the full
    # unfolding of T - E + Y_n/mu, same E-step, multipliers and mu schedule.
    dims = t.shape
    nm = len(dims)
    e = np.zeros(dims)
    ys = [np.zeros(dims) for _ in range(nm)]
    mu = mu0
    for _ in range(iters):
        zs = []
        for n in range(nm):
            g = np.moveaxis(t - e + ys[n] / mu, n, 0)
            shp = g.shape
            u, s, vt = np.linalg.svd(g.reshape(shp[0], -1), full_matrices=False)
            z = (u * np.maximum(s - lambdas[n] / mu, 0)) @ vt
            zs.append(np.moveaxis(z.reshape(shp), 0, n))
        avg = sum(t - zs[n] + ys[n] / mu for n in range(nm)) / nm
        e = np.sign(avg) * np.maximum(np.abs(avg) - 1 / (mu * nm), 0)
        for n in range(nm):
            ys[n] = ys[n] + mu * (t - zs[n] - e)
        mu = min(rho * mu, mu_max)
    return sum(zs) / nm, e


@pytest.mark.parametrize("dims,tucker", [((6, 5, 4), (2, 2, 2)), ((9, 8), (2, 2)), ((7, 2, 3), (2, 1, 2))])
def test_full_rank_bound_reduces_to_horpca(dims, tucker):
    # With R_n = I_n the active subspace is square orthogonal, U U^T = I, and
    # fold_n(U_n V_n) = SVT(G_n): PASD becomes the HoRPCA iteration of Eq. 2.
    # The matrix and (7, 2, 3) cases have R_0 = I_0 larger than the number of
    # columns P_0 of the first unfolding, so A_0 has R_0 - P_0 singular values that
    # are zero by shape, and their directions belong to the U-step's null space.
    pr = synth.planted(dims, tucker, 0.1, 21, scale="std", amp=5.0)
    t = pr.T.astype(np.float64)
    lam = O.paper_lambdas(t.shape)
    iters = 150
    p = O.Params(ranks=t.shape, lambdas=lam, stop="fixed", max_iter=iters)
    res = O.pasd(t, p)
    assert max(res.trace[-1].kept) > 0
    l_h, e_h = _horpca(t, lam, iters)
    assert np.allclose(res.L, l_h, rtol=0, atol=1e-9 * np.abs(t).max())
    assert np.allclose(res.E, e_h, rtol=0, atol=1e-9 * np.abs(t).max())


def test_default_weights_are_the_papers_setting():
    # Sec. 5.1 sets lambda_n = sqrt(max(I_n, prod_{m != n} I_m)) / N. For the 50^3 cube
    # that is sqrt(2500) / 3 = 50 / 3, the same as the (alpha_n, lambda) form with
    # alpha_n = 1/3 and lambda = 1/50 (reading 1); for a 4-way 50^4 tensor
    # sqrt(125000) / 4, and for a matrix sqrt(max(I_1, I_2)) / 2 per mode.
    assert O.paper_lambdas((50, 50, 50)) == pytest.approx([50 / 3] * 3, rel=1e-15)
    p = O.Params.from_alpha_lambda((10,) * 3, (1 / 3,) * 3, 1 / 50)
    assert list(p.lambdas) == pytest.approx(O.paper_lambdas((50, 50, 50)), rel=1e-15)
    assert O.paper_lambdas((50,) * 4) == pytest.approx([np.sqrt(125000) / 4] * 4, rel=1e-15)
    assert O.paper_lambdas((9, 400)) == pytest.approx([10.0, 10.0], rel=1e-15)


def _fold_by_index(m, n, dims):
    """fold_n written out entry by entry: Z[x] = M[x_n, j] with j the C-order index
    of x over the modes other than n (Sec. 2.1 with the column order of reading 7)."""
    z = np.empty(dims)
    for x in np.ndindex(*dims):
        j = 0
        for k, i_k in enumerate(dims):
            if k != n:
                j = j * i_k + x[k]
        z[x] = m[x[n], j]
    return z


def test_output_is_the_alpha_weighted_mean_of_the_refolds():
    # Algorithm 1's output X = sum_n alpha_n Z_n / sum_n alpha_n with unequal alpha_n,
    # against Z_n = fold_n(U_n V_n) rebuilt from the final state entry by entry. With
    # the nuclear weights lambda_n given per mode, alpha_n enters the output only: the
    # whole trajectory equals the equal-weight run bit for bit. The unweighted mean of
    # the Z_n is far from X at this (unconverged) body, so a kernel or an oracle that
    # ignored alpha would fail.
    pr = _small_problem(seed=17)
    t = pr.T.astype(np.float64)
    lam = O.paper_lambdas(t.shape)
    alpha = (0.5, 0.3, 0.2)
    iters = 120
    r_eq = O.pasd(t, O.Params(ranks=(3, 3, 3), lambdas=lam, stop="fixed", max_iter=iters))
    r_al = O.pasd(t, O.Params(ranks=(3, 3, 3), lambdas=lam, alpha=alpha, stop="fixed", max_iter=iters))
    assert max(r_al.trace[-1].kept) > 0
    for n in range(3):
        assert np.array_equal(r_al.state.U[n], r_eq.state.U[n])
        assert np.array_equal(r_al.state.V[n], r_eq.state.V[n])
    assert np.array_equal(r_al.E, r_eq.E)
    zs = [_fold_by_index(r_al.state.U[n] @ r_al.state.V[n], n, t.shape) for n in range(3)]
    want = (alpha[0] * zs[0] + alpha[1] * zs[1] + alpha[2] * zs[2]) / (alpha[0] + alpha[1] + alpha[2])
    assert np.allclose(r_al.L, want, rtol=0, atol=1e-13 * np.abs(want).max())
    mean = (zs[0] + zs[1] + zs[2]) / 3
    assert np.allclose(r_eq.L, mean, rtol=0, atol=1e-13 * np.abs(mean).max())
    assert np.linalg.norm(r_al.L - mean) > 1e-4 * np.linalg.norm(mean)
    # scaling every alpha_n by a power of two leaves X unchanged, bit for bit
    r_4 = O.pasd(t, O.Params(ranks=(3, 3, 3), lambdas=lam, alpha=tuple(4 * a for a in alpha),
                             stop="fixed", max_iter=iters))
    assert np.array_equal(r_4.L, r_al.L)


def test_alpha_lambda_form_depends_on_the_ratios_only():
    # In the (alpha_n, lambda) form lambda_n = alpha_n / lambda, so (c alpha, c lambda)
    # is the same problem: with c a power of two every lambda_n is the same double and
    # the run is the same bit for bit; unequal alpha_n change the trajectory itself.
    pr = _small_problem(seed=18)
    t = pr.T.astype(np.float64)
    alpha = (0.5, 0.3, 0.2)
    p1 = O.Params.from_alpha_lambda((3, 3, 3), alpha, 1 / 12, stop="fixed", max_iter=140)
    p2 = O.Params.from_alpha_lambda((3, 3, 3), tuple(2 * a for a in alpha), 2 / 12, stop="fixed", max_iter=140)
    assert list(p1.lambdas) == list(p2.lambdas)
    r1, r2 = O.pasd(t, p1), O.pasd(t, p2)
    assert np.array_equal(r1.L, r2.L) and np.array_equal(r1.E, r2.E)
    r_eq = O.pasd(t, O.Params.from_alpha_lambda((3, 3, 3), (1 / 3,) * 3, 1 / 12, stop="fixed", max_iter=140))
    assert [s.kept for s in r1.trace] != [s.kept for s in r_eq.trace] or not np.allclose(r1.E, r_eq.E)


def test_zero_tensor_stops_after_one_body_at_zero():
    # T = 0 is a fixed point of Algorithm 1: G = 0, so A = 0, V = 0, Z = 0, E = 0 and
    # Y stays 0; the residual is exactly zero, so the stop test holds after one body.
    for dims, ranks in (((6, 5, 4), (2, 2, 2)), ((7, 3), (3, 3))):
        res = O.pasd(np.zeros(dims), O.Params(ranks=ranks, lambdas=O.paper_lambdas(dims)))
        assert res.converged and res.iters == 1
        assert not res.L.any() and not res.E.any()
        assert res.trace[0].kept == [0] * len(dims) and res.trace[0].res_inf == 0.0
        for n, (i_n, r_n) in enumerate(zip(dims, ranks)):
            assert np.array_equal(res.state.U[n], np.eye(i_n, r_n))


def test_scale_equivariance():
    # (T, mu0, mu_max) -> (cT, mu0/c, mu_max/c) maps (L, E, Y) -> (cL, cE, Y): each
    # sub-step of Eq. 10, 13, 15 is homogeneous under this change.
    pr = _small_problem(seed=14)
    t = pr.T.astype(np.float64)
    lam = O.paper_lambdas(t.shape)
    base = O.Params(ranks=(3, 3, 3), lambdas=lam, stop="fixed", max_iter=230)
    r1 = O.pasd(t, base)
    c = 8.0
    scaled = O.Params(ranks=(3, 3, 3), lambdas=lam, stop="fixed", max_iter=230,
                      mu0=base.mu0 / c, mu_max=base.mu_max / c)
    r2 = O.pasd(c * t, scaled)
    assert [s.kept for s in r1.trace] == [s.kept for s in r2.trace]
    assert np.allclose(r2.L, c * r1.L, rtol=0, atol=1e-10 * c)
    assert np.allclose(r2.E, c * r1.E, rtol=0, atol=1e-10 * c)


def test_mode_permutation_equivariance():
    pr = _small_problem(seed=15)
    t = pr.T.astype(np.float64)
    ranks = (3, 4, 2)
    lam = (2.0, 3.0, 1.5)
    perm = (2, 0, 1)
    r1 = O.pasd(t, O.Params(ranks=ranks, lambdas=lam, stop="fixed", max_iter=200))
    tp = np.transpose(t, perm)
    r2 = O.pasd(tp, O.Params(ranks=tuple(ranks[i] for i in perm),
                             lambdas=tuple(lam[i] for i in perm), stop="fixed", max_iter=200))
    assert max(r1.trace[-1].kept) > 0
    assert np.allclose(r2.L, np.transpose(r1.L, perm), atol=1e-10)
    assert np.allclose(r2.E, np.transpose(r1.E, perm), atol=1e-10)


def test_unfolding_column_order_does_not_matter(monkeypatch):
    pr = _small_problem(seed=16)
    t = pr.T.astype(np.float64)
    p = O.Params(ranks=(3, 3, 3), lambdas=O.paper_lambdas(t.shape), stop="fixed", max_iter=220)
    r1 = O.pasd(t, p)

    def unfold_f(x, n):
        return np.moveaxis(x, n, 0).reshape(x.shape[n], -1, order="F")

    def fold_f(m, n, dims):
        dims = tuple(dims)
        rest = dims[:n] + dims[n + 1:]
        return np.moveaxis(m.reshape((dims[n],) + rest, order="F"), 0, n)

    monkeypatch.setattr(O, "unfold", unfold_f)
    monkeypatch.setattr(O, "fold", fold_f)
    r2 = O.pasd(t, p)
    assert max(r1.trace[-1].kept) > 0
    assert np.allclose(r1.L, r2.L, atol=1e-10)
    assert np.allclose(r1.E, r2.E, atol=1e-10)


def test_subspaces_stay_orthonormal():
    pr = _small_problem(seed=17)
    t = pr.T.astype(np.float64)
    p = O.Params(ranks=(3, 3, 3), lambdas=O.paper_lambdas(t.shape), stop="fixed", max_iter=250)
    st = O.init_state(t, p.ranks, p.mu0)
    for _ in range(p.max_iter):
        O.step(t, st, p)
        for u in st.U:
            assert np.allclose(u.T @ u, np.eye(u.shape[1]), atol=1e-12)


def test_recovers_planted_tensor_and_stops():
    # Planted Tucker + sparse recovery (Sec. 5.1): Algorithm 1 stops in finitely many
    # iterations (Theorem 1) and succeeds by the paper's criterion RSE <= 1e-3.
    pr = synth.cube_small(0)
    p = O.Params.from_alpha_lambda((10, 10, 10), (1 / 3,) * 3, 1 / 50, stop="inf", max_iter=1000)
    r = O.pasd(pr.T, p)
    assert r.converged and r.iters < 1000
    assert O.rse(r.L, pr.L0) < 1e-5
    assert r.trace[-1].kept == [5, 5, 5]     # the planted Tucker rank
    # recovered sparse part sits on the corrupted support
    big = np.abs(r.E.ravel()) > 1e-6 * np.abs(pr.T).max()
    assert np.mean(np.isin(np.flatnonzero(big), pr.support)) > 0.99


def test_fp32_state_floor_dense_sparse_part():
    # Not a pin of the oracle: the size of the difference any FP32-storage solver
    # must show against it. Rounding the oracle's own state (E, Y_n, U_n, V_n) to
    # float32 after every loop body moves E by more than 1e-5 relative on the
    # reduced video-shaped tensor (dense E of magnitude ~1e-2, formed from
    # differences of O(0.3) values; measured 4.0e-5) and the output L (Algorithm 1's
    # sum_n alpha_n Z_n / sum_n alpha_n from the rounded U_n, V_n) by 8.0e-6, while on
    # a planted cube with sparse outliers the same rounding stays near 1e-7. This is
    # why the GPU parity test holds the video case's E to 1e-4 and its L to 2e-5
    # (2.5 times these floors), and every sparse-E case to 1e-5.
    r32 = lambda x: x.astype(np.float32).astype(np.float64)

    def floor(pr, ranks, iters):
        T = pr.T.astype(np.float64)
        p = O.Params(ranks=ranks, lambdas=O.paper_lambdas(pr.T.shape), stop="fixed", max_iter=iters)
        exact = O.pasd(T, p)
        st = O.init_state(T, p.ranks, p.mu0)
        for _ in range(iters):
            O.step(T, st, p)
            st.E = r32(st.E)
            st.Y = [r32(y) for y in st.Y]
            st.U = [r32(u) for u in st.U]
            st.V = [r32(v) for v in st.V]
        L = O.output_low_rank([O.fold(st.U[n] @ st.V[n], n, T.shape) for n in range(T.ndim)], p.alpha)
        return (np.linalg.norm(st.E - exact.E) / np.linalg.norm(exact.E),
                np.linalg.norm(L - exact.L) / np.linalg.norm(exact.L))

    video_e, video_l = floor(synth.video(height=36, width=44, frames=40, n_rect=4, seed=3), (10, 10, 3, 5), 150)
    cube_e, cube_l = floor(synth.planted((24, 20, 16), (3, 3, 2), 0.1, 7, scale="std", amp=5.0), (4, 4, 3), 150)
    assert 1e-5 < video_e < 1e-4
    assert 2e-6 < video_l < 2e-5
    assert cube_e < 1e-6 and cube_l < 1e-6


def test_idle_start_closed_form():
    # Algorithm 1 from V_n = 0, E = 0 at the paper's mu0: while nothing is kept
    # and E stays 0, a loop body only adds mu T to every multiplier, so
    # Y_n^i = mu0 T (rho^i - 1) / (rho - 1) and G_n^i = T + Y_n^i / mu^i = g_i T.
    # Iteration i stays idle exactly while g_i sigma_max(T_(n)[:R_n]) <= lambda_n / mu^i
    # for every n (Eq. 13 with U_n = eye) and g_i max|T| <= 1 / (N mu^i) (Eq. 15).
    # The first active iteration predicted from these two tests must be the
    # oracle's, which is what the solver's idle-start skip relies on.
    pr = synth.planted((16, 14, 12), (2, 2, 2), 0.1, 5, scale="std", amp=5.0)
    T = pr.T.astype(np.float64)
    ranks = (3, 3, 3)
    p = O.Params(ranks=ranks, lambdas=O.paper_lambdas(T.shape), stop="fixed", max_iter=400)
    smax = [np.linalg.svd(O.unfold(T, n)[:ranks[n]], compute_uv=False)[0] for n in range(3)]
    tmax = float(np.abs(T).max())
    mu, c, i_a = p.mu0, 0.0, 0
    while (1 + c) * tmax <= 1 / (mu * 3) and all((1 + c) * smax[n] <= p.lambdas[n] / mu for n in range(3)):
        mn = min(p.rho * mu, p.mu_max)
        c = (c + 1) * mu / mn
        mu = mn
        i_a += 1
    assert i_a > 10
    st = O.init_state(T, ranks, p.mu0)
    for it in range(i_a + 1):
        info = O.step(T, st, p)
        if it < i_a:
            assert info.kept == [0, 0, 0] and not st.E.any()
            closed = p.mu0 * T * (p.rho ** (it + 1) - 1) / (p.rho - 1)
            for n in range(3):
                assert np.allclose(st.Y[n], closed, rtol=1e-12, atol=0)
        else:
            assert any(info.kept) or st.E.any()
