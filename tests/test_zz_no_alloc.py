"""The allocation-free mode-n product against the allocating one.

pasd_mode_product_noalloc serves callers that cannot allocate device memory
where they need the product; it keeps its Gram partial sums in a fixed scratch
array inside the library. Its results must equal pasd_mode_product's, on two
calls in a row (the second call must not see the first call's leftovers).
"""
import numpy as np
import pytest

from paper_1712_09999_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_1712_09999_gb300 import pasd as P
    return torch, P


def _case(torch, dims, mode, R, seed):
    x = synth.random_tensor(dims, seed=seed)
    pre = int(np.prod(dims[:mode])); I = dims[mode]; post = int(np.prod(dims[mode + 1:]))
    u = np.random.Generator(np.random.PCG64(seed + 1)).standard_normal((I, R)).astype(np.float32)
    return (torch.from_numpy(x).cuda(), pre, I, post, torch.from_numpy(u).cuda(), R)


def _rel(a, b):
    return float(torch_norm(a - b) / torch_norm(b))


def torch_norm(t):
    return float(t.double().norm())


def test_noalloc_equals_allocating_entry_point_twice(env):
    torch, P = env
    # first call: many CTAs; second call: fewer CTAs and another rank, so stale
    # partial sums of the first call would show up in the second Gram matrix
    for dims, mode, R, seed in (((200, 200, 200), 1, 20, 3), ((48, 40, 36), 2, 8, 4)):
        X, pre, I, post, U, R = _case(torch, dims, mode, R, seed)
        A_ref = torch.empty(pre * R * post, device="cuda")
        G_ref = torch.empty(R * R, device="cuda")
        P.pasd_mode_product(X, pre, I, post, U, R, A_ref, G_ref)
        A = torch.full_like(A_ref, float("nan"))
        G = torch.full_like(G_ref, float("nan"))
        P.pasd_mode_product_noalloc(X, pre, I, post, U, R, A, G)
        torch.cuda.synchronize()
        assert _rel(A, A_ref) <= TOL
        assert _rel(G, G_ref) <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, P = env
    # ceil(1e6 / 256) * 64 * 64 floats exceed the fixed 2^20-float scratch
    X = torch.zeros(1, device="cuda")
    A = torch.zeros(1, device="cuda")
    with pytest.raises(P.PasdError) as ei:
        P.pasd_mode_product_noalloc(X, 1000, 64, 1000, X, 64, A)
    assert ei.value.status == P.ERR_UNSUPPORTED
