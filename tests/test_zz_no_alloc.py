"""The allocation-free mode-n product against the allocating one.

pasd_mode_product_noalloc serves callers that cannot allocate device memory
where they need the product (a framework allocator that must own every device
byte, or a loop where cudaMalloc/cudaFree would synchronise the device); it
keeps its Gram partial sums in a fixed scratch array inside the library. Its
results must equal pasd_mode_product's, on two calls in a row (the second call
must not see the first call's leftovers), on the default stream and on a side
stream, and a call must not change the device's free memory.
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


CASES = (((200, 200, 200), 1, 20, 3), ((48, 40, 36), 2, 8, 4))


def test_noalloc_equals_allocating_entry_point_twice(env):
    torch, P = env
    # first call: many CTAs; second call: fewer CTAs and another rank, so stale
    # partial sums of the first call would show up in the second Gram matrix
    for dims, mode, R, seed in CASES:
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


def test_noalloc_on_a_side_stream_and_without_allocating(env):
    torch, P = env
    for dims, mode, R, seed in CASES:
        X, pre, I, post, U, R = _case(torch, dims, mode, R, seed)
        A_ref = torch.empty(pre * R * post, device="cuda")
        G_ref = torch.empty(R * R, device="cuda")
        P.pasd_mode_product(X, pre, I, post, U, R, A_ref, G_ref)
        A = torch.full_like(A_ref, float("nan"))
        G = torch.full_like(G_ref, float("nan"))
        # warm-up: loads the kernels of this rank and sets up the scratch
        P.pasd_mode_product_noalloc(X, pre, I, post, U, R, A, G)
        torch.cuda.synchronize()
        A.fill_(float("nan"))
        G.fill_(float("nan"))
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        free0, _ = torch.cuda.mem_get_info()
        P.pasd_mode_product_noalloc(X, pre, I, post, U, R, A, G, side)
        side.synchronize()          # the call is ordered on `side` only
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert _rel(A, A_ref) <= TOL
        assert _rel(G, G_ref) <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, P = env
    # the smallest shape past the fixed 2^20-float scratch: pre * post = 256 * 257
    # columns give ceil(65792 / 256) = 257 CTA partials of 64 x 64 floats; every
    # buffer has the size such a call would touch, and the outputs stay untouched
    pre, I, post, R = 256, 64, 257, 64
    assert -(-(pre * post) // 256) * R * R > 1 << 20
    X = torch.ones(pre * I * post, device="cuda")
    U = torch.ones(I * R, device="cuda")
    A = torch.full((pre * R * post,), 3.0, device="cuda")
    G = torch.full((R * R,), 5.0, device="cuda")
    A0, G0 = A.clone(), G.clone()
    with pytest.raises(P.PasdError) as ei:
        P.pasd_mode_product_noalloc(X, pre, I, post, U, R, A, G)
    assert ei.value.status == P.ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.equal(A, A0) and torch.equal(G, G0)
