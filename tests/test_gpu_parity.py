"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Acceptance (FP32 path): the number of kept singular values is identical per
mode and per iteration, and the relative Frobenius differences of L and E are
at most 1e-5; the recovery error of a converged solve is within 1e-4 of the
oracle's.
"""
import numpy as np
import pytest

from oracle import pasd_oracle as O
from paper_1712_09999_gb300 import synth
from parity_util import tie_margin

pytestmark = pytest.mark.gpu

TOL = 1e-5
STOPS = {0: "inf", 1: "fro_rel", 2: "fixed"}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_1712_09999_gb300 import pasd as P
    ctx = P.pasd_ctx_create(0)
    yield torch, P, ctx
    P.pasd_ctx_destroy(ctx)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def _gpu_solve(env, T, ranks, stop, max_iter, **kw):
    torch, P, ctx = env
    params = P.make_params(T.shape, ranks, stop=stop, max_iter=max_iter, **kw)
    plan, _ = P.pasd_plan(ctx, params)
    Td = torch.from_numpy(T).cuda()
    L = torch.empty_like(Td)
    E = torch.empty_like(Td)
    res = P.pasd_solve(plan, Td, L, E)
    trace = np.zeros((res.iters, P.TRACE_STRIDE))
    P.pasd_state_get(plan, P.STATE_TRACE, 0, trace)
    out = dict(res=res, L=L.cpu().numpy(), E=E.cpu().numpy(), trace=trace, plan=plan)
    return out


def _oracle(T, ranks, stop, max_iter, lam_pair=None):
    if lam_pair is None:
        p = O.Params(ranks=ranks, lambdas=O.paper_lambdas(T.shape), stop=STOPS[stop], max_iter=max_iter)
    else:
        alpha, lam = lam_pair
        p = O.Params.from_alpha_lambda(ranks, alpha, lam, stop=STOPS[stop], max_iter=max_iter)
    res = O.pasd(T, p)
    # the evidence that identical kept counts are not luck: no singular value on tau
    tie_margin(res.trace, p.lambdas, f"{T.shape} R={tuple(ranks)} stop={STOPS[stop]} iters={res.iters}")
    return res


def _stop_tie(ref, g_iters, tol, tmax):
    # The stop test compares a residual formed from FP32-stored tensors with tol.
    # When the oracle's residual at the earlier of the two stopping bodies lies
    # within FP32 rounding of tol (a few units of 2^-24 max|T|), stopping at
    # either body is correct: a tie, like a singular value equal to tau.
    k = min(g_iters, ref.iters)
    return abs(g_iters - ref.iters) == 1 and abs(ref.trace[k - 1].res_inf - tol) <= 4 * 2.0 ** -24 * tmax


def _check_parity(g, ref, n_modes):
    gk = g["trace"][:, 5:5 + n_modes].astype(int).tolist()
    rk = [s.kept for s in ref.trace]
    assert g["res"].iters == ref.iters
    assert gk == rk, "kept counts differ (first at %s)" % next(i for i, (a, b) in enumerate(zip(gk, rk)) if a != b)
    assert _rel(g["L"], ref.L) <= TOL
    assert _rel(g["E"], ref.E) <= TOL


@pytest.mark.parametrize("stop,iters", [(2, 150), (0, 1000)])
def test_small_cube_matches_oracle(env, stop, iters):
    pr = synth.planted((24, 20, 16), (3, 3, 2), 0.1, 7, scale="std", amp=5.0)
    ref = _oracle(pr.T, (4, 4, 3), stop, iters)
    g = _gpu_solve(env, pr.T, (4, 4, 3), stop, iters)
    _check_parity(g, ref, 3)


def test_cube50_workload_fixed_and_converged(env):
    # 50^3, Tucker core 5^3, 10% corruption U[-10,10]*std(L0), R_n = 10,
    # lambda = 1/sqrt(50*50), alpha_n = 1/3, fixed 100 iterations, then to convergence.
    pr = synth.cube_small(0)
    lp = ((1 / 3,) * 3, 1 / 50)
    kw = dict(alpha=lp[0], lam=lp[1])
    ref = _oracle(pr.T, (10,) * 3, 2, 100, lp)
    g = _gpu_solve(env, pr.T, (10,) * 3, 2, 100, **kw)
    _check_parity(g, ref, 3)
    ref = _oracle(pr.T, (10,) * 3, 0, 1000, lp)
    g = _gpu_solve(env, pr.T, (10,) * 3, 0, 1000, **kw)
    _check_parity(g, ref, 3)
    assert ref.converged and g["res"].status == 0
    assert abs(O.rse(g["L"], pr.L0) - O.rse(ref.L, pr.L0)) <= 1e-4
    assert O.rse(g["L"], pr.L0) < 1e-5


@pytest.mark.parametrize("dims,tucker,ranks", [
    ((37, 29, 23), (3, 2, 2), (5, 4, 3)),        # ragged tiles, odd contiguous mode
    ((12, 10, 3, 20), (2, 2, 2, 2), (3, 3, 2, 4)),  # 4-way with a tiny mode
    ((60, 45), (4, 4), (6, 6)),                   # matrix case (N = 2)
    ((6, 7, 5, 4, 9), (2, 2, 2, 2, 2), (2, 3, 2, 2, 3)),  # 5-way
    ((9, 8, 7), (2, 2, 2), (9, 8, 7)),            # R_n = I_n (HoRPCA case)
    # kept counts well below R_n: the M_n product runs at heights 4 and 8 of a
    # 12- or 20-row Vrot, with more split-K slices than at full height
    ((40, 36, 32), (3, 3, 3), (12, 12, 12)),
    ((64, 48, 40), (4, 4, 4), (20, 20, 20)),
    # a short mode before the last (tile 32 x 4 x 8): a thread's two element
    # groups lie half a tile apart along mode 0 instead of along mode 1
    ((48, 6, 24), (3, 2, 3), (6, 4, 6)),
])
def test_shapes_match_oracle(env, dims, tucker, ranks):
    pr = synth.planted(dims, tucker, 0.1, 3, scale="std", amp=5.0)
    ref = _oracle(pr.T, ranks, 0, 1000)
    g = _gpu_solve(env, pr.T, ranks, 0, 1000)
    _check_parity(g, ref, len(dims))


@pytest.mark.parametrize("dims,tucker,ranks", [
    ((9, 8), (2, 2), (9, 8)),              # R_0 = I_0 = 9 above P_0 = 8
    ((12, 3, 2), (2, 2, 1), (8, 3, 2)),    # R_0 = 8 above P_0 = 6, below I_0
])
def test_rank_bound_above_unfolding_columns(env, dims, tucker, ranks):
    # A_0 = U_0^T G_0 is R_0 x P_0 with R_0 > P_0: R_0 - P_0 of its singular values
    # are zero by shape, and their directions belong to the U-step's null space.
    # Fixed 200 bodies (both solves converge near 160-190 bodies, the second with its
    # last residual within 1% of tol, so a fixed count keeps the comparison free of
    # a stopping tie).
    pr = synth.planted(dims, tucker, 0.1, 3, scale="std", amp=5.0)
    ref = _oracle(pr.T, ranks, 2, 200)
    g = _gpu_solve(env, pr.T, ranks, 2, 200)
    _check_parity(g, ref, len(dims))


def test_hyperspectral_shape_matches_oracle(env):
    # Hyperspectral-shaped cube (rows, columns, bands) with salt-and-pepper noise
    # (entries replaced by 0 or 1) and an odd band count (19, padded to 20 inside
    # the solver): kept counts per iteration, stopping body, L and E.
    pr = synth.hyperspectral((24, 20, 19), (3, 3, 2), 0.10, 31)
    ref = _oracle(pr.T, (4, 4, 3), 0, 1000)
    g = _gpu_solve(env, pr.T, (4, 4, 3), 0, 1000)
    _check_parity(g, ref, 3)
    assert abs(O.rse(g["L"], pr.L0) - O.rse(ref.L, pr.L0)) <= 1e-4


def test_video_shape_matches_oracle(env):
    # Colour-video-shaped tensor (height, width, channel, frame) at reduced size:
    # rank-1 background in the frame mode, moving rectangles replacing ~4% of the
    # voxels; R = (10, 10, 3, 5) (the channel mode at R_n = I_n), the paper's
    # default lambda_n. Kept counts identical at every iteration and L within 2e-5,
    # at a fixed 150 bodies (past the activation at body 54) and at Algorithm 1's
    # stop rule (same stopping body, recovery error within 1e-4). Here E is dense at
    # the 1e-2 level (it absorbs the background's per-frame gain) and is formed from
    # differences of O(0.3) values: rounding only the FP64 oracle's state to FP32
    # after every body already moves E by 4e-5 relative and L by 8e-6
    # (tests/test_oracle_pins.py::test_fp32_state_floor_dense_sparse_part), so E is
    # held to 1e-4 and L to 2e-5, 2.5 times the FP32 storage floor of this workload
    # (measured on the GPU: 7e-6 to 1.2e-5, depending on which A-pass partial sums the
    # autotuner picks for the shape).
    # A stop one body apart is accepted only as a tie (_stop_tie), and L, E are
    # then compared with the oracle run to the GPU's stopping body.
    pr = synth.video(height=36, width=44, frames=40, n_rect=4, seed=3)
    ranks = (10, 10, 3, 5)
    for stop, iters in ((2, 150), (0, 1000)):
        ref = _oracle(pr.T, ranks, stop, iters)
        g = _gpu_solve(env, pr.T, ranks, stop, iters)
        if stop == 0:
            assert ref.converged and g["res"].status == 0
            if g["res"].iters != ref.iters:
                assert _stop_tie(ref, g["res"].iters, 1e-5, float(np.abs(pr.T).max()))
                ref = _oracle(pr.T, ranks, 2, g["res"].iters)
        gk = g["trace"][:, 5:9].astype(int).tolist()
        assert g["res"].iters == ref.iters
        assert gk == [s.kept for s in ref.trace]
        assert _rel(g["L"], ref.L) <= 2e-5
        assert _rel(g["E"], ref.E) <= 1e-4
    assert abs(O.rse(g["L"], pr.L0) - O.rse(ref.L, pr.L0)) <= 1e-4


def _gpu_state(env, plan, shape, ranks):
    torch, P, ctx = env
    N = len(shape)
    D = int(np.prod(shape))
    st = {}
    for n in range(N):
        I, R = shape[n], ranks[n]
        u = np.zeros((I, R), np.float32); P.pasd_state_get(plan, P.STATE_U, n, u)
        a = np.zeros((R, D // I), np.float32); P.pasd_state_get(plan, P.STATE_A, n, a)
        w = np.zeros((R, R), np.float32); P.pasd_state_get(plan, P.STATE_W, n, w)
        f = np.zeros(R, np.float32); P.pasd_state_get(plan, P.STATE_F, n, f)
        s = np.zeros(R, np.float32); P.pasd_state_get(plan, P.STATE_SIGMA, n, s)
        y = np.zeros(shape, np.float32); P.pasd_state_get(plan, P.STATE_Y, n, y)
        st[n] = dict(U=u.astype(np.float64), A=a.astype(np.float64), W=w.astype(np.float64),
                     F=f.astype(np.float64), sigma=s, Y=y.astype(np.float64))
    e = np.zeros(shape, np.float32); P.pasd_state_get(plan, P.STATE_E, 0, e)
    mu = np.zeros(1, np.float64); P.pasd_state_get(plan, P.STATE_MU, 0, mu)
    kept = np.zeros(N, np.int32); P.pasd_state_get(plan, P.STATE_KEPT, 0, kept)
    return st, e.astype(np.float64), float(mu[0]), kept.tolist()


def test_full_size_single_step_parity(env):
    # 200^3 workload (Tucker core 10^3, 20% corruption U[-1,1]*max|L0|, R_n = 20,
    # lambda = 1/200, alpha = 1/3): run the GPU past the activation, hand its state
    # to the oracle, and compare one loop body of each.
    torch, P, ctx = env
    pr = synth.cube_200(1)
    T = pr.T
    shape, ranks = T.shape, (20, 20, 20)
    params = P.make_params(shape, ranks, alpha=(1 / 3,) * 3, lam=1 / 200, stop=P.STOP_FIXED_ITERS,
                           max_iter=1000)
    plan, _ = P.pasd_plan(ctx, params)
    Td = torch.from_numpy(T).cuda()
    P.pasd_begin(plan, Td)
    P.pasd_iterate(plan, 115)
    torch.cuda.synchronize()
    st, e, mu, kept = _gpu_state(env, plan, shape, ranks)
    assert max(kept) > 0, "state is still idle"
    t64 = T.astype(np.float64)
    ost = O.State(U=[], V=[], null=[], E=e, Y=[], mu=mu, k=115)
    for n in range(3):
        s = st[n]
        k = kept[n]
        ost.U.append(s["U"])
        ost.V.append((s["W"] * s["F"]) @ (s["W"].T @ s["A"]))
        ost.null.append(s["W"][:, k:])
        ost.Y.append(s["Y"])
    p = O.Params.from_alpha_lambda(ranks, (1 / 3,) * 3, 1 / 200, stop="fixed", max_iter=1000)
    info = O.step(t64, ost, p)
    P.pasd_iterate(plan, 1)
    torch.cuda.synchronize()
    st2, e2, mu2, kept2 = _gpu_state(env, plan, shape, ranks)
    assert kept2 == info.kept
    assert mu2 == pytest.approx(ost.mu, rel=1e-12)
    assert _rel(e2, ost.E) <= TOL
    for n in range(3):
        s = st2[n]
        z = O.fold(s["U"] @ ((s["W"] * s["F"]) @ (s["W"].T @ s["A"])), n, shape)
        assert _rel(z, info.Z[n]) <= TOL
        # multipliers: compare to their own scale
        assert np.max(np.abs(s["Y"] - ost.Y[n])) <= 1e-4 * np.max(np.abs(ost.Y[n])) + 1e-6
        k = info.kept[n]
        assert np.allclose(s["sigma"][:k], info.sigma[n][:k], rtol=1e-4)
        assert np.allclose(s["U"].T @ s["U"], np.eye(ranks[n]), atol=1e-5)
    P.pasd_plan_destroy(plan)


def test_full_size_trajectory_matches_oracle_golden(env):
    # 200^3 workload solved to relative residual 1e-6 in the benchmark's launch
    # configuration, against the oracle's solve stored by
    # tests/golden/make_cube200_trajectory.py: identical kept counts at every
    # iteration and the same stopping iteration; the infinity-norm residual within
    # FP32 rounding of |T| (a few ulps of max|T| per term); L and E at 512 seeded
    # positions within the 1e-5 relative Frobenius bound (estimated on the sample).
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "cube200_trajectory.json")
    gold = json.load(open(path))
    torch, P, ctx = env
    pr = synth.cube_200(1)
    T = pr.T
    params = P.make_params(T.shape, tuple(gold["ranks"]), alpha=tuple(gold["alpha"]), lam=gold["lambda"],
                           stop=P.STOP_FRO_REL, tol=gold["tol"], max_iter=1000)
    plan, _ = P.pasd_plan(ctx, params)
    Td = torch.from_numpy(T).cuda()
    L = torch.empty_like(Td)
    E = torch.empty_like(Td)
    res = P.pasd_solve(plan, Td, L, E)
    trace = np.zeros((res.iters, P.TRACE_STRIDE))
    P.pasd_state_get(plan, P.STATE_TRACE, 0, trace)
    gk = trace[:, 5:8].astype(int).tolist()
    first = next((i + 1 for i, (a, b) in enumerate(zip(gk, gold["kept"])) if a != b), None)
    assert first is None, "kept counts differ first at iteration %d: %s vs %s" % (
        first, gk[first - 1], gold["kept"][first - 1])
    assert res.iters == gold["iters"] and res.status == 0
    tmax = float(np.abs(T).max())
    ri = np.asarray(gold["res_inf"])
    assert np.all(np.abs(trace[:, 1] - ri) <= 1e-4 * ri + 1e-6 * tmax)
    idx = np.asarray(gold["sample_index"])
    lg = L.reshape(-1)[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    eg = E.reshape(-1)[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    assert _rel(lg, np.asarray(gold["L_sample"])) <= TOL
    assert _rel(eg, np.asarray(gold["E_sample"])) <= TOL
    assert float(torch.linalg.vector_norm(L.double())) == pytest.approx(gold["L_fro"], rel=TOL)
    assert float(torch.linalg.vector_norm(E.double())) == pytest.approx(gold["E_fro"], rel=TOL)
    P.pasd_plan_destroy(plan)


@pytest.mark.parametrize("case", ["small_fixed", "small_converged", "cube50"])
def test_idle_skip_matches_oracle(env, case):
    # PASD_F_SKIP_IDLE replaces the idle bodies after the first by their closed
    # form; the trace (kept counts per iteration), the iteration count and L, E
    # must still be the oracle's, and bodies must actually have been skipped.
    _, P, _ = env
    if case == "cube50":
        pr = synth.cube_small(0)
        ranks, stop, iters, lp = (10,) * 3, 2, 100, ((1 / 3,) * 3, 1 / 50)
        kw = dict(alpha=lp[0], lam=lp[1])
    else:
        pr = synth.planted((24, 20, 16), (3, 3, 2), 0.1, 7, scale="std", amp=5.0)
        ranks, lp, kw = (4, 4, 3), None, {}
        stop, iters = (2, 150) if case == "small_fixed" else (0, 1000)
    ref = _oracle(pr.T, ranks, stop, iters, lp)
    g = _gpu_solve(env, pr.T, ranks, stop, iters, flags=P.F_SKIP_IDLE, **kw)
    _check_parity(g, ref, 3)
    first_active = next(i for i, s in enumerate(ref.trace) if any(s.kept))
    assert 0 < g["res"].skipped < first_active
    # replaced bodies are recorded like computed idle ones
    tr = g["trace"]
    assert np.all(tr[:first_active, 5:8] == 0)
    assert np.array_equal(tr[:, 0], np.arange(1, g["res"].iters + 1))


def test_idle_skip_full_size_trajectory(env):
    # the 200^3 workload with the idle-start skip against the oracle's stored solve
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "cube200_trajectory.json")
    gold = json.load(open(path))
    torch, P, ctx = env
    pr = synth.cube_200(1)
    params = P.make_params(pr.T.shape, tuple(gold["ranks"]), alpha=tuple(gold["alpha"]), lam=gold["lambda"],
                           stop=P.STOP_FRO_REL, tol=gold["tol"], max_iter=1000, flags=P.F_SKIP_IDLE)
    plan, _ = P.pasd_plan(ctx, params)
    Td = torch.from_numpy(pr.T).cuda()
    L = torch.empty_like(Td)
    E = torch.empty_like(Td)
    res = P.pasd_solve(plan, Td, L, E)
    trace = np.zeros((res.iters, P.TRACE_STRIDE))
    P.pasd_state_get(plan, P.STATE_TRACE, 0, trace)
    assert trace[:, 5:8].astype(int).tolist() == gold["kept"]
    assert res.iters == gold["iters"] and res.status == 0
    first_active = next(i for i, k in enumerate(gold["kept"]) if any(k))
    assert 50 <= res.skipped < first_active
    idx = torch.from_numpy(np.asarray(gold["sample_index"])).cuda()
    assert _rel(L.reshape(-1)[idx].cpu().numpy().astype(np.float64), np.asarray(gold["L_sample"])) <= TOL
    assert _rel(E.reshape(-1)[idx].cpu().numpy().astype(np.float64), np.asarray(gold["E_sample"])) <= TOL
    P.pasd_plan_destroy(plan)


MIXED_TOL = 1e-3


def _check_mixed(g, ref, n_modes):
    # mixed precision (tensor-core TF32-split V-step products): the same kept
    # counts at every iteration and the same stopping iteration, L and E within 1e-3
    gk = g["trace"][:, 5:5 + n_modes].astype(int).tolist()
    rk = [s.kept for s in ref.trace]
    assert g["res"].iters == ref.iters
    assert gk == rk, "kept counts differ (first at %s)" % next(i for i, (a, b) in enumerate(zip(gk, rk)) if a != b)
    assert _rel(g["L"], ref.L) <= MIXED_TOL
    assert _rel(g["E"], ref.E) <= MIXED_TOL


@pytest.mark.parametrize("stop,iters", [(2, 150), (0, 1000)])
def test_mixed_small_cube_matches_oracle(env, stop, iters):
    _, P, _ = env
    pr = synth.planted((24, 20, 16), (3, 3, 2), 0.1, 7, scale="std", amp=5.0)
    ref = _oracle(pr.T, (4, 4, 3), stop, iters)
    g = _gpu_solve(env, pr.T, (4, 4, 3), stop, iters, precision=P.PREC_MIXED)
    _check_mixed(g, ref, 3)


@pytest.mark.parametrize("dims,tucker,ranks", [
    ((40, 36, 32), (3, 3, 3), (12, 12, 12)),
    ((64, 48, 40), (4, 4, 4), (20, 20, 20)),
    ((12, 10, 3, 20), (2, 2, 2, 2), (3, 3, 2, 4)),
])
def test_mixed_shapes_match_oracle(env, dims, tucker, ranks):
    _, P, _ = env
    pr = synth.planted(dims, tucker, 0.1, 3, scale="std", amp=5.0)
    ref = _oracle(pr.T, ranks, 0, 1000)
    g = _gpu_solve(env, pr.T, ranks, 0, 1000, precision=P.PREC_MIXED)
    _check_mixed(g, ref, len(dims))


def test_mixed_full_size_trajectory_matches_oracle_golden(env):
    # the 200^3 workload solved with mixed precision against the oracle's stored
    # solve: identical kept counts per iteration, same stopping iteration, sampled
    # L and E within 1e-3, recovery error within 1e-4 of the FP64 solve's
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "cube200_trajectory.json")
    gold = json.load(open(path))
    torch, P, ctx = env
    pr = synth.cube_200(1)
    params = P.make_params(pr.T.shape, tuple(gold["ranks"]), alpha=tuple(gold["alpha"]), lam=gold["lambda"],
                           stop=P.STOP_FRO_REL, tol=gold["tol"], max_iter=1000, precision=P.PREC_MIXED)
    plan, _ = P.pasd_plan(ctx, params)
    Td = torch.from_numpy(pr.T).cuda()
    L = torch.empty_like(Td)
    E = torch.empty_like(Td)
    res = P.pasd_solve(plan, Td, L, E)
    trace = np.zeros((res.iters, P.TRACE_STRIDE))
    P.pasd_state_get(plan, P.STATE_TRACE, 0, trace)
    assert trace[:, 5:8].astype(int).tolist() == gold["kept"]
    assert res.iters == gold["iters"] and res.status == 0
    idx = torch.from_numpy(np.asarray(gold["sample_index"])).cuda()
    assert _rel(L.reshape(-1)[idx].cpu().numpy().astype(np.float64), np.asarray(gold["L_sample"])) <= MIXED_TOL
    assert _rel(E.reshape(-1)[idx].cpu().numpy().astype(np.float64), np.asarray(gold["E_sample"])) <= MIXED_TOL
    L0 = torch.from_numpy(pr.L0).cuda()
    rse = float(torch.linalg.vector_norm(L.double() - L0) / torch.linalg.vector_norm(L0))
    assert abs(rse - gold["rse"]) <= 1e-4
    P.pasd_plan_destroy(plan)


def test_multiplier_bound_and_orthonormality_on_gpu(env):
    # ||sum_n Y_n||_inf <= 1 (App. A) and U_n^T U_n = I along a GPU run.
    torch, P, ctx = env
    pr = synth.planted((40, 36, 32), (3, 3, 3), 0.15, 9, scale="std", amp=5.0)
    shape, ranks = pr.T.shape, (5, 5, 4)
    plan, _ = P.pasd_plan(ctx, P.make_params(shape, ranks, stop=P.STOP_FIXED_ITERS, max_iter=400))
    Td = torch.from_numpy(pr.T).cuda()
    P.pasd_begin(plan, Td)
    for _ in range(8):
        P.pasd_iterate(plan, 25)
        torch.cuda.synchronize()
        st, e, mu, kept = _gpu_state(env, plan, shape, ranks)
        ysum = sum(st[n]["Y"] for n in range(3))
        slack = 1e-4 + 64 * np.finfo(np.float32).eps * mu * np.abs(pr.T).max()
        assert np.max(np.abs(ysum)) <= 1.0 + slack
        for n in range(3):
            assert np.allclose(st[n]["U"].T @ st[n]["U"], np.eye(ranks[n]), atol=1e-5)
    P.pasd_plan_destroy(plan)


def test_stepwise_and_host_paths_equal_solve(env):
    torch, P, ctx = env
    pr = synth.planted((30, 26, 22), (3, 3, 3), 0.1, 12, scale="std", amp=5.0)
    shape, ranks = pr.T.shape, (4, 4, 4)
    params = P.make_params(shape, ranks, stop=P.STOP_INF_ABS, max_iter=1000)
    plan, _ = P.pasd_plan(ctx, params)
    Td = torch.from_numpy(pr.T).cuda()
    L1 = torch.empty_like(Td); E1 = torch.empty_like(Td)
    r1 = P.pasd_solve(plan, Td, L1, E1)
    # stepwise
    L2 = torch.empty_like(Td); E2 = torch.empty_like(Td)
    P.pasd_begin(plan, Td)
    P.pasd_iterate(plan, r1.iters + 20)     # bodies after the stop rule are skipped
    r2 = P.pasd_finish(plan, L2, E2)
    assert r2.iters == r1.iters
    assert torch.equal(L1, L2) and torch.equal(E1, E2)
    # host buffers
    Lh = np.zeros(shape, np.float32); Eh = np.zeros(shape, np.float32)
    r3 = P.pasd_solve_host(plan, np.ascontiguousarray(pr.T), Lh, Eh)
    assert r3.iters == r1.iters
    assert np.array_equal(Lh, L1.cpu().numpy()) and np.array_equal(Eh, E1.cpu().numpy())
    P.pasd_plan_destroy(plan)


@pytest.mark.parametrize("mode", ["fp32", "fp32_skip", "mixed_skip"])
def test_served_results_equal_alone(env, mode):
    # Continuous batching: solves submitted together overlap on the device; each
    # result equals the same solve run alone (FP32, FP32 with the idle-start skip,
    # mixed precision with the skip).
    torch, P, ctx = env
    prec = P.PREC_MIXED if mode.startswith("mixed") else P.PREC_FP32
    flags = P.F_SKIP_IDLE if mode.endswith("skip") else 0
    probs = [synth.planted(d, (3, 3, 3), 0.1, 20 + i, scale="std", amp=5.0)
             for i, d in enumerate([(32, 30, 28), (40, 24, 36), (28, 28, 28), (50, 20, 30)])]
    plans, alone, bufs, skipped = [], [], [], []
    for pr in probs:
        plan, _ = P.pasd_plan(ctx, P.make_params(pr.T.shape, (4, 4, 4), max_iter=1000, precision=prec, flags=flags))
        Td = torch.from_numpy(pr.T).cuda()
        L = torch.empty_like(Td); E = torch.empty_like(Td)
        r0 = P.pasd_solve(plan, Td, L, E)
        skipped.append(r0.skipped)
        alone.append((L.clone(), E.clone()))
        L.zero_(); E.zero_()
        plans.append(plan)
        bufs.append((Td, L, E))
    torch.cuda.synchronize()
    tickets = [P.pasd_submit(ctx, plans[i], *bufs[i]) for i in range(len(probs))]
    import time
    t0 = time.time()
    pending = set(tickets)
    results = {}
    while pending and time.time() - t0 < 60:
        for t in list(pending):
            st, r = P.pasd_poll(ctx, t)
            if st != P.PENDING:
                results[t] = (st, r)
                pending.discard(t)
        time.sleep(0.001)
    assert not pending
    for i, t in enumerate(tickets):
        st, r = results[t]
        assert st == P.OK
        assert r.latency_s > 0
        assert r.skipped == skipped[i] and (skipped[i] > 0) == bool(flags)
        # every solve here advances in the batched executor (mixed precision with
        # its tensor-core A-pass launched per solve inside the batched body)
        assert r.batched == 1
        assert torch.equal(bufs[i][1], alone[i][0]) and torch.equal(bufs[i][2], alone[i][1])
    for plan in plans:
        P.pasd_plan_destroy(plan)


def test_first_solve_on_a_plan_is_ordered_after_its_setup(env):
    # A plan's device memory is allocated and cleared on its first use. The clear
    # must be complete before the solve starts on a stream that does not wait for
    # the legacy default stream (the served path's streams, or a caller's
    # non-blocking stream), even while other work holds that default stream: here
    # a bounded spin kernel of about 10 ms. Results equal solves on used plans.
    torch, P, ctx = env
    probs = [synth.planted((100, 100, 100), (6, 6, 6), 0.1, 40 + i, scale="std", amp=5.0) for i in range(3)]
    ref = []
    for pr in probs:
        plan, _ = P.pasd_plan(ctx, P.make_params(pr.T.shape, (8, 8, 8), max_iter=1000, flags=P.F_SKIP_IDLE))
        Td = torch.from_numpy(pr.T).cuda()
        L = torch.empty_like(Td); E = torch.empty_like(Td)
        r = P.pasd_solve(plan, Td, L, E)
        ref.append((r.iters, L.clone(), E.clone(), Td))
        P.pasd_plan_destroy(plan)
    torch.cuda.synchronize()

    # served path: two solves on never-used plans
    fresh = [P.pasd_plan(ctx, P.make_params(pr.T.shape, (8, 8, 8), max_iter=1000, flags=P.F_SKIP_IDLE))[0]
             for pr in probs[:2]]
    outs = [(torch.empty_like(ref[i][3]), torch.empty_like(ref[i][3])) for i in range(2)]
    torch.cuda.synchronize()
    torch.cuda._sleep(20_000_000)
    tickets = [P.pasd_submit(ctx, fresh[i], ref[i][3], *outs[i]) for i in range(2)]
    import time
    t0 = time.time()
    results = {}
    while len(results) < 2 and time.time() - t0 < 60:
        for t in tickets:
            if t not in results:
                st, r = P.pasd_poll(ctx, t)
                if st != P.PENDING:
                    results[t] = (st, r)
        time.sleep(0.001)
    torch.cuda.synchronize()
    assert len(results) == 2
    for i, t in enumerate(tickets):
        st, r = results[t]
        assert st == P.OK and r.iters == ref[i][0]
        assert torch.equal(outs[i][0], ref[i][1]) and torch.equal(outs[i][1], ref[i][2])
    for plan in fresh:
        P.pasd_plan_destroy(plan)

    # stepwise on a caller's non-blocking stream, on a never-used plan
    plan, _ = P.pasd_plan(ctx, P.make_params(probs[2].T.shape, (8, 8, 8), max_iter=1000, flags=P.F_SKIP_IDLE))
    L = torch.empty_like(ref[2][3]); E = torch.empty_like(ref[2][3])
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    torch.cuda._sleep(20_000_000)
    P.pasd_begin(plan, ref[2][3], side)
    P.pasd_iterate(plan, ref[2][0], side)
    r = P.pasd_finish(plan, L, E, side)
    torch.cuda.synchronize()
    assert r.iters == ref[2][0]
    assert torch.equal(L, ref[2][1]) and torch.equal(E, ref[2][2])
    P.pasd_plan_destroy(plan)


def test_a_plan_belongs_to_the_served_path_until_it_retires(env):
    # While a served solve of a plan is queued or running, the entry points that
    # touch the plan's state refuse it with BUSY (destroying it included); once
    # the ticket has been polled to a final status the plan is the caller's again.
    torch, P, ctx = env
    pr = synth.planted((100, 100, 100), (6, 6, 6), 0.1, 50, scale="std", amp=5.0)
    params = P.make_params(pr.T.shape, (8, 8, 8), stop=P.STOP_FIXED_ITERS, max_iter=1000)
    plan, _ = P.pasd_plan(ctx, params)
    Td = torch.from_numpy(pr.T).cuda()
    L = torch.empty_like(Td); E = torch.empty_like(Td)
    torch.cuda.synchronize()
    ticket = P.pasd_submit(ctx, plan, Td, L, E)     # 1000 bodies: tens of milliseconds
    host = np.zeros(1, np.float64)
    for call in (lambda: P.pasd_plan_destroy(plan), lambda: P.pasd_solve(plan, Td, L, E),
                 lambda: P.pasd_begin(plan, Td), lambda: P.pasd_iterate(plan, 1),
                 lambda: P.pasd_finish(plan, L, E), lambda: P.pasd_state_get(plan, P.STATE_MU, 0, host)):
        with pytest.raises(P.PasdError) as err:
            call()
        assert err.value.status == P.ERR_BUSY
    import time
    t0 = time.time()
    while True:
        st, r = P.pasd_poll(ctx, ticket)
        if st != P.PENDING or time.time() - t0 > 60:
            break
        time.sleep(0.001)
    assert st == P.OK and r.iters == 1000
    served_L = L.clone()
    res = P.pasd_solve(plan, Td, L, E)
    assert res.iters == 1000 and torch.equal(L, served_L)
    P.pasd_plan_destroy(plan)


def test_invalid_and_nonfinite_inputs(env):
    torch, P, ctx = env
    with pytest.raises(P.PasdError) as ei:
        P.pasd_plan(ctx, P.make_params((10, 8, 6), (4, 9, 2)))    # R_2 > I_2
    assert ei.value.status == P.ERR_INVALID_ARG
    with pytest.raises(P.PasdError) as ei:
        P.pasd_plan(ctx, P.make_params((10, 8, 6), (4, 4, 2), rho=0.9))
    assert ei.value.status == P.ERR_INVALID_ARG
    pr = synth.planted((20, 18, 16), (2, 2, 2), 0.1, 2, scale="std", amp=5.0)
    t = pr.T.copy()
    t[3, 4, 5] = np.nan
    plan, _ = P.pasd_plan(ctx, P.make_params(t.shape, (3, 3, 3), max_iter=50))
    Td = torch.from_numpy(t).cuda()
    L = torch.full_like(Td, 7.0); E = torch.full_like(Td, 7.0)
    with pytest.raises(P.PasdError) as ei:
        P.pasd_solve(plan, Td, L, E)
    assert ei.value.status == P.ERR_NONFINITE
    assert bool(torch.all(L == 7.0)) and bool(torch.all(E == 7.0))   # outputs untouched
    P.pasd_plan_destroy(plan)
