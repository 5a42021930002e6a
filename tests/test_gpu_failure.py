"""Failure detection on the GPU without a fault: a bounded device-side wait that nothing
satisfies expires, the library reports POND_ERR_TIMEOUT, and the CUDA context stays usable
(a solver created afterwards steps and matches the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2203_05477_gb300 as pond  # noqa: E402
from paper_2203_05477_gb300 import inputs as I  # noqa: E402
from tests.common import max_rel, oracle_for  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("polls", [1, 1000])
def test_bounded_wait_expires_and_the_context_survives(polls):
    assert pond.pond_wait_timeout_check(polls, None) == pond.POND_ERR_TIMEOUT
    assert b"expired" in pond.pond_last_error()
    pb = I.sod_400()
    kw = dict(tau=1e-5, cfl=0.5, fixed_iters=3, max_iter=8)
    s = pond.Solver(pb, precision="fp64", **kw)
    s.set_primitive()
    s.step(5)
    d = s.sync()
    assert d["status"] == pond.POND_OK and d["steps"] == 5
    o = oracle_for(pb, **kw)
    o.step(5)
    (r, _, _, E), _ = s.moments(totals=False)
    ro, _, _, Eo = o.conserved()
    assert max_rel(r, ro) <= 1e-12 and max_rel(E, Eo) <= 1e-12
    s.close()
