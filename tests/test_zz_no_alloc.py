"""pond_mlp_gradient_noalloc: the gradient of the learned-predictor network computed with
the library's fixed device scratch instead of a cudaMalloc, for callers that cannot
allocate device memory.  Checked through the C ABI against pond_mlp_gradient on two calls
in a row (the scratch is reused and must not carry state from one call to the next)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2203_05477_gb300 as pond  # noqa: E402
from oracle import gauge_mlp as G  # noqa: E402

pytestmark = pytest.mark.gpu

MAX_ROWS = 8192  # POND_MLP_NOALLOC_MAX_ROWS


def _abi():
    lib = pond._load()
    fn = lib.pond_mlp_gradient_noalloc
    vp = ctypes.c_void_p
    fn.restype = ctypes.c_int
    fn.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int64, vp, vp, vp]
    return lib, fn


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, 52), dtype=np.float32)
    X[:, :34] = rng.standard_normal((n, 34)).astype(np.float32)
    X[:, 48:51] = rng.standard_normal((n, 3)).astype(np.float32)
    p = G.init_params(seed).astype(np.float32)
    return torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()


def _noalloc(fn, p, X, n):
    grad = torch.full((G.NPARAMS,), float("nan"), dtype=torch.float32, device="cuda")
    loss = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
    st = fn(p.data_ptr(), X.data_ptr(), 52, X.data_ptr(), 52, n, grad.data_ptr(), loss.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    assert st == pond.POND_OK, pond._load().pond_last_error()
    return float(loss.item()), grad.cpu().numpy()


def test_noalloc_gradient_matches_the_allocating_entry_point():
    lib, fn = _abi()
    for call, (n, seed) in enumerate([(1000, 21), (MAX_ROWS, 22)]):
        p, X = _inputs(n, seed)
        loss_ref, g_ref = pond.mlp_gradient(p, X, X)
        g_ref = g_ref.cpu().numpy()
        loss, g = _noalloc(fn, p, X, n)
        # the same tolerance as the tensor-core gradient test: 3e-2 of each tensor's scale
        assert loss == pytest.approx(loss_ref, rel=1e-2), call
        for lo, hi in [(G.O_W1, G.O_B1), (G.O_B1, G.O_W2), (G.O_W2, G.O_B2), (G.O_B2, G.O_W3), (G.O_W3, G.O_B3),
                       (G.O_B3, G.NPARAMS)]:
            scale = max(np.abs(g_ref[lo:hi]).max(), 1e-12)
            assert np.abs(g[lo:hi] - g_ref[lo:hi]).max() <= 3e-2 * scale, (call, lo)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib, fn = _abi()
    p, X = _inputs(MAX_ROWS + 1, 23)
    grad = torch.zeros(G.NPARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    st = fn(p.data_ptr(), X.data_ptr(), 52, X.data_ptr(), 52, MAX_ROWS + 1, grad.data_ptr(), loss.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    assert st == pond.POND_ERR_INVALID_ARG
    assert b"exceeds" in lib.pond_last_error()
