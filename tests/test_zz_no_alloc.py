"""pond_mlp_gradient_noalloc: the gradient of the learned-predictor network computed with
the library's fixed device scratch instead of a cudaMalloc, for callers that cannot
allocate device memory (a framework's caching allocator holds the device, the
device-wide synchronization of cudaMalloc/cudaFree is not allowed, or a failed allocation
could not be handled).

Checked through the C ABI on consecutive calls of decreasing size (so rows left in the
shared scratch by a larger earlier call are present and must not leak into a smaller one):
against the FP64 reference network with the kernels' bfloat16 rounding points, at the
tolerance of the tensor-core gradient test; against pond_mlp_gradient, which runs the same
kernels on a cudaMalloc'ed scratch, where the gradient is deterministic (each weight
gradient is one tensor-core accumulation in a fixed order) and only the loss, a sum of
FP32 atomics, may differ in its last bits; and with the device's free memory unchanged
across the calls."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2203_05477_gb300 as pond  # noqa: E402
from oracle import gauge_mlp as G  # noqa: E402

pytestmark = pytest.mark.gpu

MAX_ROWS = 8192  # POND_MLP_NOALLOC_MAX_ROWS
BLOCKS = [(G.O_W1, G.O_B1), (G.O_B1, G.O_W2), (G.O_W2, G.O_B2), (G.O_B2, G.O_W3), (G.O_W3, G.O_B3),
          (G.O_B3, G.NPARAMS)]


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
    return p, X


def _call(fn, p, X, n, grad, loss):
    st = fn(p.data_ptr(), X.data_ptr(), 52, X.data_ptr(), 52, n, grad.data_ptr(), loss.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    assert st == pond.POND_OK, pond._load().pond_last_error()


def test_noalloc_gradient_matches_reference_and_allocating_entry_point():
    lib, fn = _abi()
    cases = [(MAX_ROWS, 22), (1000, 21), (257, 23)]
    dev = [(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()) for p, X in (_inputs(n, s) for n, s in cases)]
    grads = [torch.full((G.NPARAMS,), float("nan"), dtype=torch.float32, device="cuda") for _ in cases]
    losses = [torch.full((1,), float("nan"), dtype=torch.float32, device="cuda") for _ in cases]
    # a first call loads the library's module (and with it the scratch array) if nothing has yet
    _call(fn, dev[-1][0], dev[-1][1], cases[-1][0], grads[-1], losses[-1])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k, (n, _) in enumerate(cases):
        _call(fn, dev[k][0], dev[k][1], n, grads[k], losses[k])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    for k, (n, seed) in enumerate(cases):
        p, X = _inputs(n, seed)
        g = grads[k].cpu().numpy()
        loss = float(losses[k].item())
        # against the FP64 reference network (bfloat16 at the kernels' rounding points): the
        # tolerance of the tensor-core gradient test, 3e-2 of each tensor's scale
        lref, gref = G.loss_and_grad(p.astype(np.float64), X.astype(np.float64), X[:, 48:51].astype(np.float64),
                                     quantize=True)
        assert loss == pytest.approx(lref, rel=1e-2), k
        for lo, hi in BLOCKS:
            scale = max(np.abs(gref[lo:hi]).max(), 1e-12)
            assert np.abs(g[lo:hi] - gref[lo:hi]).max() <= 3e-2 * scale, (k, lo)
        # against the allocating entry point: the same kernels on the same inputs
        loss_a, g_a = pond.mlp_gradient(dev[k][0], dev[k][1], dev[k][1])
        g_a = g_a.cpu().numpy()
        assert loss == pytest.approx(loss_a, rel=1e-5), k
        for lo, hi in BLOCKS:
            scale = max(np.abs(g_a[lo:hi]).max(), 1e-12)
            assert np.abs(g[lo:hi] - g_a[lo:hi]).max() <= 1e-6 * scale, (k, lo)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib, fn = _abi()
    p, X = _inputs(MAX_ROWS + 1, 23)
    p, X = torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()
    grad = torch.zeros(G.NPARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    st = fn(p.data_ptr(), X.data_ptr(), 52, X.data_ptr(), 52, MAX_ROWS + 1, grad.data_ptr(), loss.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    assert st == pond.POND_ERR_INVALID_ARG
    assert b"exceeds" in lib.pond_last_error()
