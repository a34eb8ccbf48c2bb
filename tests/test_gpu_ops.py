"""GPU checks of the standalone mode-n product (the V-step's A_n = U_n^T X_(n)
and its Gram matrix) against FP64 numpy on the same inputs."""
import numpy as np
import pytest

from paper_1712_09999_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_1712_09999_gb300 import pasd as P
    return torch, P


def _ref(x, pre, I, post, u):
    x3 = x.reshape(pre, I, post).astype(np.float64)
    a = np.einsum("ir,aib->arb", u.astype(np.float64), x3)
    a2 = a.transpose(1, 0, 2).reshape(u.shape[1], -1)
    return a, a2 @ a2.T


@pytest.mark.parametrize("dims,mode,R", [
    ((200, 200, 200), 0, 20), ((200, 200, 200), 1, 20), ((200, 200, 200), 2, 20),
    ((37, 29, 23), 1, 8), ((37, 29, 23), 2, 12),          # odd strides: 4-byte copy paths
    ((64, 50, 33), 0, 64), ((300, 7), 1, 4), ((5, 1000), 0, 4),
    ((12, 10, 3, 20), 2, 4),
])
def test_mode_product_matches_fp64(env, dims, mode, R):
    torch, P = env
    x = synth.random_tensor(dims, seed=31)
    pre = int(np.prod(dims[:mode])); I = dims[mode]; post = int(np.prod(dims[mode + 1:]))
    rng = np.random.Generator(np.random.PCG64(5))
    u = rng.standard_normal((I, R)).astype(np.float32)
    if I >= R:
        u = np.linalg.qr(u.astype(np.float64))[0].astype(np.float32)
    X = torch.from_numpy(x).cuda()
    U = torch.from_numpy(u).cuda()
    A = torch.empty(pre * R * post, device="cuda")
    Gm = torch.empty(R * R, device="cuda")
    P.pasd_mode_product(X, pre, I, post, U, R, A, Gm)
    a_ref, g_ref = _ref(x, pre, I, post, u)
    a = A.cpu().numpy().reshape(pre, R, post)
    g = Gm.cpu().numpy().reshape(R, R)
    assert np.linalg.norm(a - a_ref) <= 1e-5 * np.linalg.norm(a_ref)
    assert np.linalg.norm(g - g_ref) <= 1e-5 * np.linalg.norm(g_ref)


def test_mode_product_rejects_unsupported_rank(env):
    torch, P = env
    X = torch.zeros(4 * 5 * 6, device="cuda")
    U = torch.zeros(5 * 3, device="cuda")
    A = torch.zeros(4 * 3 * 6, device="cuda")
    with pytest.raises(P.PasdError) as ei:
        P.pasd_mode_product(X, 4, 5, 6, U, 3, A)
    assert ei.value.status == P.ERR_UNSUPPORTED
