"""The slab-sharded form of Algorithm 1 against the single-process oracle (CPU only).

The sharded body splits the tensor along one mode over several ranks and meets
only through the exchanges its module lists. It must reproduce the oracle's
trajectory: the same kept counts in every body, the same stopping body, and L, E
equal up to the rounding of the two routes. The two routes take the small
factors differently (LAPACK SVD of the whole matrix against a tall-skinny QR),
so they agree to eps * kappa, with kappa the condition number of G_n V_n^T on
its range: a direction the SVT has just kept has a singular value barely above
zero there (kappa reaches about 2e8 on the ragged case below, so 1e-7 bounds L
and E; the well-conditioned cases agree to about 1e-11).
"""
import os
import socket
import threading

import numpy as np
import pytest

from oracle import pasd_oracle as O
from oracle import pasd_sharded as S
from paper_1712_09999_gb300 import synth

TOL = 1e-7


class ThreadComm(S.Comm):
    """Ranks as threads of one process; every collective combines the ranks' values in
    rank order, so every rank gets the same bits."""

    def __init__(self, rank, world, shared):
        super().__init__(rank, world)
        self.shared = shared

    def _all(self, x, combine):
        slots = self.shared["slots"]
        slots[self.rank] = x
        self.shared["barrier"].wait()
        out = slots[0]
        for v in slots[1:]:
            out = combine(out, v)
        out = np.array(out, copy=True)
        self.shared["barrier"].wait()
        return out

    def _sum(self, x):
        return self._all(x, lambda a, b: a + b)

    def _max(self, x):
        return float(self._all(np.array(x), np.maximum))

    def _gather(self, x):
        return self._all(x, lambda a, b: np.concatenate([a, b], 0))


def _slab(T, m, lo, hi):
    index = [slice(None)] * T.ndim
    index[m] = slice(lo, hi)
    return T[tuple(index)]


def _problem(dims, tucker, ranks, seed=7, max_iter=600):
    pr = synth.planted(dims, tucker, 0.1, seed, scale="std", amp=5.0)
    T = pr.T.astype(np.float64)
    return T, O.Params(ranks=ranks, lambdas=O.paper_lambdas(dims), max_iter=max_iter)


class SkippingComm(ThreadComm):
    """A planted mistake: one kind of all-reduce keeps each rank's own part."""

    def __init__(self, rank, world, shared, skip):
        super().__init__(rank, world, shared)
        self.skip = skip

    def sum(self, x, kind):
        if kind == self.skip:
            return np.ascontiguousarray(x, dtype=np.float64)
        return super().sum(x, kind)

    def gather(self, x, kind):
        if kind == self.skip:
            return np.ascontiguousarray(x, dtype=np.float64)
        return super().gather(x, kind)


def _run_threads(T, p, m, world, make_comm=ThreadComm, check=True):
    shared = {"slots": [None] * world, "barrier": threading.Barrier(world)}
    bounds = S.slab_bounds(T.shape[m], world)
    out, errors = [None] * world, []

    def rank_main(r):
        try:
            lo, hi = bounds[r]
            comm = make_comm(r, world, shared)
            out[r] = (S.pasd_sharded(_slab(T, m, lo, hi), T.shape, m, lo, hi, p, comm), comm)
        except BaseException as exc:  # noqa: BLE001 - reported below
            errors.append(exc)
            shared["barrier"].abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    if check:
        assert not errors, errors
    return out, errors


def _expected_elements(dims, ranks, m, trace):
    want = {"init": 1}
    before = [0] * len(dims)
    for info in trace:
        for kind, count in S.exchange_elements(dims, ranks, m, before).items():
            want[kind] = want.get(kind, 0) + count
        before = info.kept
    return want


def _check(ref, L, E, res, comm_elements, dims, ranks, m):
    assert res.iters == ref.iters and res.converged == ref.converged
    assert [i.kept for i in res.trace] == [i.kept for i in ref.trace]
    assert np.linalg.norm(L - ref.L) <= TOL * np.linalg.norm(ref.L)
    assert np.linalg.norm(E - ref.E) <= TOL * np.linalg.norm(ref.E)
    assert abs(res.trace[-1].res_inf - ref.trace[-1].res_inf) <= TOL * np.abs(ref.L).max()
    assert res.trace[-1].objective == pytest.approx(ref.trace[-1].objective, rel=TOL)
    assert dict(comm_elements) == _expected_elements(dims, ranks, m, ref.trace)


@pytest.mark.parametrize("dims,tucker,ranks,m,world", [
    ((9, 7, 6), (2, 2, 2), (4, 3, 3), 0, 3),
    ((9, 7, 6), (2, 2, 2), (4, 3, 3), 1, 3),
    ((9, 7, 6), (2, 2, 2), (4, 3, 3), 2, 3),
    ((8, 6, 2), (2, 2, 1), (3, 3, 2), 2, 3),       # R_m = I_m, one rank holds no slab
    ((7, 6, 5, 4), (2, 2, 2, 2), (3, 3, 3, 2), 2, 3),
    ((12, 9), (2, 2), (3, 3), 0, 2),               # matrix case
    ((12, 3, 2), (2, 2, 1), (8, 3, 2), 1, 2),      # R_0 = 8 above P_0 = 6
])
def test_sharded_matches_oracle(dims, tucker, ranks, m, world):
    T, p = _problem(dims, tucker, ranks)
    ref = O.pasd(T, p)
    out, _ = _run_threads(T, p, m, world)
    L = np.concatenate([o[0].L for o in out], axis=m)
    E = np.concatenate([o[0].E for o in out], axis=m)
    for res, comm in out:
        _check(ref, L, E, res, comm.elements, dims, ranks, m)


@pytest.mark.parametrize("skip,m", [("M", 0), ("rfac", 0), ("A", 0), ("rfac", 2), ("proj", 2)])
def test_a_missing_exchange_is_caught(skip, m):
    """Each exchange is needed: leaving one out changes the trajectory (or breaks it)."""
    T, p = _problem((9, 7, 6), (2, 2, 2), (4, 3, 3), max_iter=200)
    ref = O.pasd(T, p)
    out, errors = _run_threads(T, p, m, 2, lambda r, w, sh: SkippingComm(r, w, sh, skip), check=False)
    if errors:
        return
    L = np.concatenate([o[0].L for o in out], axis=m)
    kept = [i.kept for i in out[0][0].trace]
    assert kept != [i.kept for i in ref.trace] or np.linalg.norm(L - ref.L) > 1e-3 * np.linalg.norm(ref.L)


def test_single_rank_is_the_whole_problem():
    """With one rank the slab is the tensor and nothing is exchanged between ranks."""
    T, p = _problem((9, 7, 6), (2, 2, 2), (4, 3, 3), max_iter=120)
    ref = O.pasd(T, p)
    res = S.pasd_sharded(T, T.shape, 1, 0, 7, p, S.Comm())
    assert [i.kept for i in res.trace] == [i.kept for i in ref.trace]
    assert np.linalg.norm(res.L - ref.L) <= TOL * max(np.linalg.norm(ref.L), 1e-300)


def test_exchange_volume_at_200_cube():
    """Values one rank contributes per body at 200^3, R_n = 20, slab along mode 0 with
    every direction kept: 2 x (200 x 20 + 20^2) for the other modes, 2 x 20^2 R factors,
    20 x 40000 for A_0 and 5 stop scalars; about 3.2 MB in FP32."""
    e = S.exchange_elements((200, 200, 200), (20, 20, 20), 0, (20, 20, 20))
    assert e == {"M": 8000, "rfac": 1200, "A": 800000, "stop": 5}
    e = S.exchange_elements((200, 200, 200), (20, 20, 20), 0, (12, 20, 20))
    assert e["rfac"] == 1600 and e["proj"] == 400


def test_slab_bounds():
    assert S.slab_bounds(7, 3) == [(0, 3), (3, 5), (5, 7)]
    assert S.slab_bounds(2, 3) == [(0, 1), (1, 2), (2, 2)]
    with pytest.raises(ValueError):
        S.pasd_sharded(np.zeros((2, 3, 4)), (4, 3, 4), 0, 0, 3, O.Params(ranks=(1, 1, 1), lambdas=(1, 1, 1)),
                       S.Comm())


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, m, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        T, p = _problem((10, 9, 7), (2, 2, 2), (4, 4, 3))
        lo, hi = S.slab_bounds(T.shape[m], world)[rank]
        comm = S.DistComm(dist)
        res = S.pasd_sharded(_slab(T, m, lo, hi), T.shape, m, lo, hi, p, comm)
        q.put((rank, res.L, res.E, res.iters, [i.kept for i in res.trace], dict(comm.elements),
               [u.copy() for n, u in enumerate(res.state.U) if n != m]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_sharded_over_two_gloo_ranks():
    """Two processes over torch.distributed (gloo), slab along mode 1 (5 + 4 rows)."""
    pytest.importorskip("torch")
    import multiprocessing as mp
    m, world = 1, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, world, port, m, q)) for r in range(world)]
    for proc in procs:
        proc.start()
    got = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for proc in procs:
        proc.join(timeout=60)
        assert proc.exitcode == 0
    T, p = _problem((10, 9, 7), (2, 2, 2), (4, 4, 3))
    ref = O.pasd(T, p)
    L = np.concatenate([g[1] for g in got], axis=m)
    E = np.concatenate([g[2] for g in got], axis=m)
    assert np.linalg.norm(L - ref.L) <= TOL * np.linalg.norm(ref.L)
    assert np.linalg.norm(E - ref.E) <= TOL * np.linalg.norm(ref.E)
    want = _expected_elements(T.shape, p.ranks, m, ref.trace)
    for g in got:
        assert g[3] == ref.iters
        assert g[4] == [i.kept for i in ref.trace]
        assert g[5] == want
    # the factors every rank holds whole are the same bits on both ranks
    for u0, u1 in zip(got[0][6], got[1][6]):
        assert np.array_equal(u0, u1)
