"""The learned face-gauge predictor: tensor-core forward and backward against the FP64
reference network (same bfloat16 rounding points), training, and what the trained network
changes in the solver (corrector passes per face; results within the FP32 tolerance)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2203_05477_gb300 as pond  # noqa: E402
from oracle import gauge_mlp as G  # noqa: E402
from paper_2203_05477_gb300 import inputs as I  # noqa: E402
from tests.common import gpu_primitive, rel_l1  # noqa: E402

pytestmark = pytest.mark.gpu


def batch(n, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, pond.MLP_PAIR_STRIDE), dtype=np.float32)
    X[:, :34] = rng.standard_normal((n, 34)).astype(np.float32)
    X[:, 33] = 1.0
    X[:, 48:51] = rng.standard_normal((n, 3)).astype(np.float32)
    return X


@pytest.mark.parametrize("n", [1, 128, 300])
def test_forward_matches_reference(n):
    p = G.init_params(5).astype(np.float32)
    X = batch(n, 6)
    out = pond.mlp_forward(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    ref, _ = G.forward(p.astype(np.float64), X.astype(np.float64), quantize=True)
    # FP32 accumulation against FP64: a hidden activation may round to the other bfloat16
    # neighbour (2^-8 relative); bound the output error by 1% of its scale
    scale = np.abs(ref).max()
    assert np.abs(out - ref).max() <= 1e-2 * scale, np.abs(out - ref).max() / scale


@pytest.mark.parametrize("n", [130, 1000])
def test_gradient_matches_reference(n):
    p = G.init_params(7).astype(np.float32)
    X = batch(n, 8)
    loss, g = pond.mlp_gradient(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(), torch.from_numpy(X).cuda())
    g = g.cpu().numpy()
    lref, gref = G.loss_and_grad(p.astype(np.float64), X.astype(np.float64), X[:, 48:51].astype(np.float64), quantize=True)
    assert loss == pytest.approx(lref, rel=1e-2)
    for lo, hi in [(G.O_W1, G.O_B1), (G.O_B1, G.O_W2), (G.O_W2, G.O_B2), (G.O_B2, G.O_W3), (G.O_W3, G.O_B3), (G.O_B3, G.NPARAMS)]:
        scale = max(np.abs(gref[lo:hi]).max(), 1e-12)
        assert np.abs(g[lo:hi] - gref[lo:hi]).max() <= 3e-2 * scale, (lo, np.abs(g[lo:hi] - gref[lo:hi]).max() / scale)


def test_training_fits_a_smooth_target():
    n = 8192
    X = batch(n, 9)
    rng = np.random.default_rng(10)
    A = rng.standard_normal((34, 3)).astype(np.float32) * 0.2
    X[:, 48:51] = np.tanh(X[:, :34] @ A)
    pb = I.quadrants_2d(16, seed=0)
    s = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2)
    losses = s.gauge_train(torch.from_numpy(X).cuda(), epochs=30, batch=1024, lr=3e-3)
    assert losses[-1] < 0.1 * losses[0], losses


def test_learned_predictor_in_the_solver():
    """Collect pairs from the plain FP32 solver on one seed, train on the GPU, then run
    another seed with and without the learned predictor.  The corrector still decides
    convergence: the learned run stays within 1e-4 relative L1 of the FP64 oracle, the bound
    of the plain FP32 run, and the passes per face of both runs are reported."""
    from tests.common import oracle_for
    train_pb = I.quadrants_2d(256, seed=1)
    s = pond.Solver(train_pb, precision="fp32", tau=1e-5, cfl=0.2)
    s.set_primitive()
    pairs = s.gauge_collect(200, cap=400_000, every=2)
    assert pairs.shape[0] > 10_000
    perm = torch.randperm(pairs.shape[0], device=pairs.device)
    losses = s.gauge_train(pairs[perm].contiguous(), epochs=8, batch=4096, lr=2e-3)
    assert losses[-1] < losses[0]
    params = s.gauge_params()
    s.close()

    def run(pb, learned, steps):
        g = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2)
        g.set_primitive()
        if learned:
            g.set_gauge_params(params)
            g.gauge_enable(True)
        g.step(steps)
        d = g.sync()
        assert d["status"] == pond.POND_OK, d
        out = (gpu_primitive(g), d["face_iters"] / d["face_solves"], d["nonconverged"])
        g.close()
        return out

    big = I.quadrants_2d(256, seed=2)
    _, pass0, nc0 = run(big, False, 150)
    _, pass1, nc1 = run(big, True, 150)
    print("passes per face: plain %.4f learned %.4f; non-converged faces %d / %d" % (pass0, pass1, nc0, nc1))
    # 98-99% of faces converge in one pass from the previous frame; the gated prediction
    # must not cost passes
    assert pass1 <= 1.03 * pass0

    # accuracy: the learned run is held to the plain FP32 run's bound, 1e-4 relative L1
    # against the FP64 oracle with the same stopping rule, on draws whose corrector
    # converges nearly everywhere (the oracle has 24 and 11 faces in 40 steps that reach the
    # pass limit; a Mach-3 quadrant draw has 1000-4000, where any start other than the
    # oracle's own ends elsewhere within the method's stopping-point envelope)
    for pb in (I.quadrants_2d(48, seed=6, mach_max=1.0), I.smooth_periodic(2, 48, 48, seed=2, amp=0.15)):
        os_ = oracle_for(pb, tau=1e-5, cfl=0.2, tol=1e-6)
        os_.step(40)
        assert os_.stats()["fallbacks"] == 0 and os_.stats()["nonconverged"] <= 30
        ro, uo, vo, po = os_.primitive()
        so = np.hypot(uo, vo)
        for learned in (False, True):
            (r, u, v, p), _, _ = run(pb, learned, 40)
            err = (rel_l1(r, ro), rel_l1(p, po), np.abs(np.hypot(u, v) - so).sum() / so.sum())
            assert max(err) < 1e-4, (learned, err)


def _run_quadrants(params, steps, gate=None, trust=None, max_iter=16):
    pb = I.quadrants_2d(48, seed=0)
    g = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2, max_iter=max_iter)
    g.set_primitive()
    if params is not None:
        g.set_gauge_params(params)
        g.gauge_enable(True, gate=gate, trust=trust)
    g.step(steps)
    d = g.sync()
    out = gpu_primitive(g), d
    g.close()
    return out


def test_a_biased_network_cannot_move_the_solution():
    """A network that predicts the same wrong correction for every face (zero weights, output
    bias (0.3, -0.2, 0.1) in units of sqrt(T) and log T, inside the trust radius) only moves
    where the corrector starts.  Faces that converge end where the corrector's fixed point
    is, and the others are solved again from the previous half step's frame.  On this draw
    (1500 faces cycle without converging), a face next to a limit cycle can also settle
    from another start, so the run is held to the method's own stopping-point envelope: how
    far the plain run moves when max_iter changes by one (measured alongside)."""
    p = np.zeros(G.NPARAMS, dtype=np.float32)
    p[G.O_B3:G.O_B3 + 3] = (0.3, -0.2, 0.1)
    (r0, u0, v0, p0), d0 = _run_quadrants(None, 30)
    env_r = env_p = 0.0
    for mi in (15, 17):
        (re_, _, _, pe_), _ = _run_quadrants(None, 30, max_iter=mi)
        env_r, env_p = max(env_r, rel_l1(re_, r0)), max(env_p, rel_l1(pe_, p0))
    (r1, u1, v1, p1), d1 = _run_quadrants(p, 30, gate=0.0)
    assert d1["status"] == pond.POND_OK and d1["nonphysical"] == 0
    assert d1["face_iters"] > d0["face_iters"]   # the wrong start costs passes
    dr, dp = rel_l1(r1, r0), rel_l1(p1, p0)
    print("biased network: rho %.2e p %.2e; envelope rho %.2e p %.2e" % (dr, dp, env_r, env_p))
    assert dr <= max(3e-5, 2 * env_r) and dp <= max(3e-5, 2 * env_p), (dr, dp, env_r, env_p)
    # beyond the trust radius the prediction is not used at all: the run is the plain one.
    # The learned instantiation of the face kernel is separate code, whose FP32 arithmetic the
    # compiler may contract differently (a mul-add fused or not), so the bound is FP32 rounding:
    # three orders below what a used prediction moves (above) and the same corrector passes
    p[G.O_B3:G.O_B3 + 3] = (3.0, -2.0, 1.0)
    (r2, u2, v2, p2), d2 = _run_quadrants(p, 30, gate=0.0)
    assert rel_l1(r2, r0) <= 1e-6 and rel_l1(p2, p0) <= 1e-6
    assert abs(d2["face_iters"] - d0["face_iters"]) <= 1e-3 * d0["face_iters"]


def test_gauge_blob_round_trip_and_learned_option():
    pb = I.quadrants_2d(32, seed=0)
    a = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2)
    p = G.init_params(11).astype(np.float32)
    a.set_gauge_params(p)
    blob = a.gauge_save()
    b = pond.Solver(pb, precision="fp32", tau=1e-5, cfl=0.2)
    b.gauge_load(blob)
    assert np.array_equal(b.gauge_params(), p)
    with pytest.raises(pond.PondError):
        b.gauge_load(b"POND" + blob[4:100])
