"""Pins for the oracle's velocity sets (Table I, Eq. wi)."""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1_d1q4.txt")


def _table1():
    nodes, weights, TL = [], [], None
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] == "TL":
            TL = float(parts[1])
            continue
        ev = {"sqrt": math.sqrt}
        nodes.append(eval(parts[0], {"__builtins__": {}}, ev))
        weights.append(eval(parts[1], {"__builtins__": {}}, ev))
    order = np.argsort(nodes)
    return np.array(nodes)[order], np.array(weights)[order], TL


def test_d1q4_matches_table1():
    c, w, TL = O.lattice(1)
    cn, wn, TLn = _table1()
    assert TL == TLn
    np.testing.assert_allclose(c[:, 0], cn, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, wn, rtol=0, atol=1e-16)


def test_d1q4_is_gauss_hermite_rule():
    c, w, _ = O.lattice(1)
    c = c[:, 0]
    # nodes are the roots of He_4(x) = x^4 - 6x^2 + 3
    np.testing.assert_allclose(c ** 4 - 6 * c ** 2 + 3, 0.0, atol=1e-13)
    # exact Gaussian moments (k-1)!! for even k up to degree 7, and not at degree 8
    exact = [1, 0, 1, 0, 3, 0, 15, 0]
    for k, e in enumerate(exact):
        assert abs(np.dot(w, c ** k) - e) < 1e-13, k
    assert abs(np.dot(w, c ** 8) - 105.0) > 1.0  # 81 on the lattice


def test_d2q16_is_tensor_product():
    c2, w2, TL = O.lattice(2)
    c1, w1, _ = O.lattice(1)
    assert c2.shape == (16, 2) and TL == 1.0
    for i in range(16):
        m = int(np.argmin(np.abs(c1[:, 0] - c2[i, 0])))
        n = int(np.argmin(np.abs(c1[:, 0] - c2[i, 1])))
        assert abs(w2[i] - w1[m] * w1[n]) < 1e-16
    # isotropy up to third order (needed by third-order Grad): sum W c_a c_b = delta_ab
    M2 = np.einsum("i,ia,ib->ab", w2, c2, c2)
    np.testing.assert_allclose(M2, np.eye(2), atol=1e-14)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w2, c2, c2, c2, c2)
    iso = lambda a, b, c, d: (a == b) * (c == d) + (a == c) * (b == d) + (a == d) * (b == c)
    for idx in np.ndindex(2, 2, 2, 2):
        assert abs(M4[idx] - iso(*idx)) < 1e-13


@pytest.mark.parametrize("kind,a,b,want", [
    (0, 1.0, 3.0, 2 * 3.0 / 4.0),      # van Leer: 2ab/(a+b)
    (0, -2.0, -2.0, -2.0),
    (0, 1.0, -1.0, 0.0),
    (0, 0.0, 5.0, 0.0),
    (0, 0.0, 0.0, 0.0),
    (1, 1.0, 3.0, 1.0),                 # minmod
    (1, -4.0, -2.0, -2.0),
    (1, 2.0, -1.0, 0.0),
])
def test_limiters_closed_form(kind, a, b, want):
    assert O.limiter(kind, a, b) == pytest.approx(want, abs=1e-15)
