"""Pins of the oracle's lattice (Sec. 2.2-2.3) against quadrature facts that do
not come from the oracle: numpy's Gauss-Hermite rule and Gaussian moments."""
import itertools
import math

import numpy as np
import pytest

import oracle


def test_d3q19_velocity_groups_and_opposites():
    c, w, opp = oracle.velocity_set()
    assert c.shape == (19, 3)
    assert len({tuple(v) for v in c}) == 19
    n = (c * c).sum(axis=1)
    # Sec. 2.3: one rest velocity, six faces, twelve edges
    assert (n == 0).sum() == 1 and (n == 1).sum() == 6 and (n == 2).sum() == 12
    for q in range(19):
        assert (c[opp[q]] == -c[q]).all()
    # weights 1/3, 1/18, 1/36 by group (Sec. 2.3)
    for q in range(19):
        assert w[q] == {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[int(n[q])]


def test_gauss_hermite_d1q3_and_tensor_weights():
    # Sec. 2.2: D1Q3 abscissae (-sqrt3, 0, sqrt3), weights (1/6, 2/3, 1/6)
    x, wt = np.polynomial.hermite_e.hermegauss(3)
    wt = wt / math.sqrt(2 * math.pi)
    assert np.allclose(np.sort(x), [-math.sqrt(3), 0, math.sqrt(3)], atol=1e-14)
    w1 = dict(zip(np.round(x / math.sqrt(3)).astype(int), wt))
    assert np.allclose([w1[-1], w1[0], w1[1]], [1 / 6, 2 / 3, 1 / 6], atol=1e-15)
    # D3Q27 weights of Sec. 2.3 are the tensor products of the 1D weights
    d3q27 = {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}
    for cv in itertools.product((-1, 0, 1), repeat=3):
        prod = w1[cv[0]] * w1[cv[1]] * w1[cv[2]]
        assert prod == pytest.approx(d3q27[sum(a * a for a in cv)], rel=1e-14)
    # and D2Q9 (4/9, 1/9, 1/36) likewise
    d2q9 = {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}
    for cv in itertools.product((-1, 0, 1), repeat=2):
        assert w1[cv[0]] * w1[cv[1]] == pytest.approx(d2q9[sum(a * a for a in cv)], rel=1e-14)


def _gauss_moment(k, var):
    # E[X^k] for X ~ N(0, var)
    if k % 2:
        return 0.0
    return var ** (k // 2) * float(np.prod(np.arange(k - 1, 0, -2))) if k else 1.0


def test_d3q19_quadrature_exact_to_degree_five():
    """Sec. 2.2: D3Q19 integrates polynomials up to degree 5 exactly against the
    Gaussian weight with theta = c_s^2 = 1/3 (lattice units)."""
    c, w, _ = oracle.velocity_set()
    for e in itertools.product(range(6), repeat=3):
        if sum(e) > 5:
            continue
        lattice = float((w * np.prod(c.astype(float) ** np.array(e), axis=1)).sum())
        exact = np.prod([_gauss_moment(k, 1 / 3) for k in e])
        assert lattice == pytest.approx(exact, abs=1e-15), e
    # ... but not to degree 6: the fourth-order isotropy fails for c_x^2 c_y^2 c_z^2
    lattice = float((w * np.prod(c.astype(float) ** 2, axis=1)).sum())
    assert lattice == 0.0 and _gauss_moment(2, 1 / 3) ** 3 > 0
