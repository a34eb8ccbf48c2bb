"""The seeded input generators deliver the recipes stated for each workload (CPU only).

These pin the inputs, not the method: the planted tensors have the stated
multilinear rank and Haar factors, the corruption covers exactly the stated
number of entries with the stated values, and the video, hyperspectral,
batched and serving recipes hold. Fixed seeds make every input reproducible.
"""
import numpy as np
import pytest

from paper_1712_09999_gb300 import synth


def _unfold_rank(x, n, tol=1e-9):
    m = np.moveaxis(x, n, 0).reshape(x.shape[n], -1)
    s = np.linalg.svd(m, compute_uv=False)
    return int(np.sum(s > tol * s[0]))


def test_haar_factors_are_orthonormal_with_positive_r_diagonal():
    # q comes from the Gaussian draw G = q (d R) with d R upper triangular and a
    # positive diagonal (the sign fix that makes the QR factor exactly Haar), so
    # q^T G, with G redrawn from the same seed, is that triangular factor.
    for seed, (rows, cols) in enumerate(((9, 4), (20, 20), (50, 3))):
        q = synth.haar_orthonormal(np.random.Generator(np.random.PCG64(seed)), rows, cols)
        g = np.random.Generator(np.random.PCG64(seed)).standard_normal((rows, cols))
        assert np.allclose(q.T @ q, np.eye(cols), atol=1e-12)
        rt = q.T @ g
        assert np.allclose(np.tril(rt, -1), 0.0, atol=1e-12)
        assert np.all(np.diag(rt) > 0)
        assert np.allclose(q @ rt, g, atol=1e-12)


def test_haar_factors_are_rotation_invariant_in_distribution():
    # The first column of a Haar factor is uniform on the sphere: its coordinates have
    # mean 0 and second moment 1/rows, and no coordinate is preferred.
    rng = np.random.Generator(np.random.PCG64(1))
    rows = 6
    cols = np.array([synth.haar_orthonormal(rng, rows, 2)[:, 0] for _ in range(20000)])
    assert np.abs(cols.mean(axis=0)).max() < 0.02
    assert np.allclose((cols ** 2).mean(axis=0), 1.0 / rows, atol=0.01)


@pytest.mark.parametrize("dims,tucker,rho,scale", [
    ((24, 20, 16), (3, 3, 2), 0.10, "std"),
    ((30, 30, 30), (5, 4, 3), 0.20, "max"),
    ((10, 12, 8, 6), (2, 3, 2, 2), 0.05, "none"),
])
def test_planted_tensor_recipe(dims, tucker, rho, scale):
    pr = synth.planted(dims, tucker, rho, 5, scale=scale, amp=2.0)
    total = int(np.prod(dims))
    # exact corruption count, positions without replacement
    assert pr.support.size == int(np.floor(rho * total)) == np.unique(pr.support).size
    assert np.count_nonzero(pr.E0) == pr.support.size
    # the low-rank part has the stated multilinear rank
    for n, r in enumerate(tucker):
        assert _unfold_rank(pr.L0, n) == r
    # values U[-amp, amp], scaled as stated
    unit = {"none": 1.0, "std": float(np.std(pr.L0)), "max": float(np.max(np.abs(pr.L0)))}[scale]
    vals = pr.E0.reshape(-1)[pr.support] / unit
    assert np.abs(vals).max() <= 2.0 and np.abs(vals).max() > 1.5
    # T is L0 + E0 rounded to FP32
    assert pr.T.dtype == np.float32
    assert np.array_equal(pr.T, (pr.L0 + pr.E0).astype(np.float32))
    # reproducible from the seed
    assert np.array_equal(synth.planted(dims, tucker, rho, 5, scale=scale, amp=2.0).T, pr.T)


def test_planted_device_recipe_on_the_cpu():
    torch = pytest.importorskip("torch")
    T, L0 = synth.planted_device((20, 18, 16), (3, 2, 2), 0.15, 9, torch.device("cpu"))
    total = 20 * 18 * 16
    assert int((T != L0).sum()) == int(0.15 * total)
    for n, r in enumerate((3, 2, 2)):
        assert _unfold_rank(L0.double().numpy(), n, tol=1e-5) == r
    assert float((T - L0).abs().max()) <= 1.0


def test_hyperspectral_recipe():
    pr = synth.hyperspectral((24, 20, 19), (3, 3, 2), 0.10, 31)
    total = 24 * 20 * 19
    assert pr.L0.min() == 0.0 and pr.L0.max() == 1.0          # min-max scaled
    assert pr.support.size == int(np.floor(0.10 * total))
    hit = pr.T.reshape(-1)[pr.support]
    assert set(np.unique(hit)) <= {0.0, 1.0}                   # salt and pepper
    ones = float(np.mean(hit == 1.0))
    assert 0.4 < ones < 0.6
    for n, r in enumerate((3, 3, 2)):
        # min-max scaling adds a constant: rank at most r + 1 per unfolding
        assert _unfold_rank(pr.L0, n) <= r + 1


def test_video_recipe():
    pr = synth.video(height=36, width=44, frames=40, n_rect=4, seed=3)
    assert pr.T.shape == (36, 44, 3, 40)
    # background rank 1 along the frame mode, within [0, 1.05]
    assert _unfold_rank(pr.L0, 3) == 1
    assert pr.L0.min() >= 0.0 and pr.L0.max() <= 1.05 + 1e-12
    # foreground replaces pixels: E0 = T - L0, zero elsewhere, a few percent of voxels
    cover = np.count_nonzero(np.abs(pr.E0) > 1e-7) / pr.E0.size
    assert 0.005 < cover < 0.2


def test_batched_and_serving_mixes():
    specs = synth.batch_mix()
    assert len(specs) == 64
    rand, hyper = specs[:56], specs[56:]
    for sp in rand:
        assert all(32 <= d <= 160 for d in sp.dims) and all(3 <= r <= 15 for r in sp.tucker)
        assert sp.rank_bounds == tuple(min(d, int(1.2 * r)) for d, r in zip(sp.dims, sp.tucker))
        assert 0.05 <= sp.rho <= 0.30 and sp.kind == "planted"
    for sp in hyper:
        assert sp.dims == (128, 128, 191) and sp.tucker[2] == 4 and sp.kind == "hyperspectral"
    reqs = synth.serving_mix(200)
    sides = np.array([sp.dims[0] for sp in reqs])
    assert sides.min() >= 32 and sides.max() <= 256
    # log-uniform: the median side is near sqrt(32 * 256) = 90.5
    assert 70 < np.median(sides) < 115
    for sp in reqs:
        assert all(3 <= r <= 20 for r in sp.tucker) and 0.05 <= sp.rho <= 0.30
        assert sp.rank_bounds == tuple(min(sp.dims[0], int(1.2 * r)) for r in sp.tucker)


def test_poisson_arrivals():
    arr = synth.poisson_arrivals(200.0, 20000, seed=5)
    assert np.all(np.diff(arr) > 0)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert gaps.mean() == pytest.approx(1 / 200.0, rel=0.03)
    assert gaps.std() == pytest.approx(1 / 200.0, rel=0.05)   # exponential: std = mean
