"""Pins of the oracle's D3Q27 lattice (Sec. 2.3; the comparison stencil of the
paper) against quadrature facts, the moment-matching construction, Table 1,
conservation, the textbook D2Q9 step, the Poiseuille closed form and the
paper's statement that D3Q27 has no spurious transverse currents (Sec. 5.1)."""
import itertools
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from oracle import construction as cons
from tests.test_oracle_step import _d2q9_run


def test_d3q27_set_and_tensor_weights():
    c, w, opp = oracle.velocity_set(27)
    assert c.shape == (27, 3) and len({tuple(v) for v in c}) == 27
    x, wt = np.polynomial.hermite_e.hermegauss(3)
    w1 = dict(zip(np.round(x / math.sqrt(3)).astype(int), wt / math.sqrt(2 * math.pi)))
    for q in range(27):
        assert (c[opp[q]] == -c[q]).all()
        assert w[q] == pytest.approx(w1[c[q, 0]] * w1[c[q, 1]] * w1[c[q, 2]], rel=1e-14)
    # degree-6 moment that D3Q19 misses
    assert float((w * np.prod(c.astype(float) ** 2, axis=1)).sum()) == pytest.approx(1 / 27, rel=1e-14)


def test_d3q27_equilibrium_is_the_construction():
    """Sec. 3.1: on D3Q27 the moment matching gives Eq. 14 (second order)."""
    vels, polys = cons.constructed_equilibrium("D3Q27")
    c, _, _ = oracle.velocity_set(27)
    index = {tuple(int(a) for a in v): q for q, v in enumerate(c)}
    rng = np.random.default_rng(4)
    for _ in range(10):
        rho = 1 + rng.uniform(-0.05, 0.05)
        u = rng.uniform(-0.1, 0.1, 3)
        for kind in (oracle.STANDARD, oracle.IMPROVED):
            f = oracle.equilibrium(kind, np.array([rho]), u.reshape(3, 1), stencil=27)[0]
            for v, p in zip(vels, polys):
                exact = float(cons.evaluate(p, Fr(float(rho)), 1, [Fr(float(a)) for a in u]))
                assert f[index[v]] == pytest.approx(exact, abs=1e-15)


@pytest.mark.parametrize("coll", [oracle.SRT, oracle.TRT])
def test_d3q27_collision_conserves(coll):
    a = (1e-3, -2e-3, 5e-4)
    cfg = oracle.Config(1, 1, 1, collision=coll, tau=0.7, accel=a, stencil=27)
    c, _, _ = oracle.velocity_set(27)
    rng = np.random.default_rng(2)
    f = oracle.init(cfg, np.array([[[1.02]]]), np.array([0.04, -0.03, 0.02]).reshape(3, 1, 1, 1))
    f = f + rng.uniform(-1e-3, 1e-3, f.shape)
    f1 = oracle.step(cfg, f)
    assert f1.sum() == pytest.approx(f.sum(), abs=1e-15)
    assert np.allclose(c.T @ f1.reshape(27) - c.T @ f.reshape(27), a, atol=1e-16)


@pytest.mark.parametrize("coll", [oracle.SRT, oracle.TRT])
def test_d3q27_projects_onto_textbook_d2q9(coll):
    """Grouping D3Q27 by (c_x, c_y) gives D2Q9 for any u_z (its moments with
    e_z = 0 are the truncated Maxwellian ones)."""
    nx, ny = 9, 7
    accel = (3e-4, -1e-4)
    cfg = oracle.Config(nx, ny, 1, collision=coll, tau=0.7, accel=(accel[0], accel[1], 0.0),
                        walls=(False, True, False), stencil=27)
    rng = np.random.default_rng(6)
    rho = 1 + rng.uniform(-0.02, 0.02, (1, ny, nx))
    u = rng.uniform(-0.05, 0.05, (3, 1, ny, nx))
    r3, u3 = oracle.run(cfg, rho, u, 12)
    r2, vx, vy = _d2q9_run(rho[0], u[0, 0], u[1, 0], 0.7, 3 / 16, coll == oracle.TRT, accel, True, 12)
    assert np.abs(r3[0] - r2).max() < 1e-14
    assert np.abs(u3[0, 0] - vx).max() < 1e-14 and np.abs(u3[1, 0] - vy).max() < 1e-14


def test_d3q27_poiseuille_trt_exact():
    H, a, tau = 12, 1e-5, 0.7
    nu = (tau - 0.5) / 3
    cfg = oracle.Config(1, H, 1, collision=oracle.TRT, tau=tau, accel=(a, 0, 0), walls=(False, True, False),
                        stencil=27)
    f = oracle.step(cfg, oracle.init(cfg, np.ones(cfg.shape), np.zeros((3,) + cfg.shape)), 20000)
    _, u = oracle.moments(cfg, f)
    y = np.arange(H)
    exact = a / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    assert np.abs(u[0, 0, :, 0] - exact).max() / exact.max() < 1e-9


def test_d3q27_no_transverse_velocity_in_cross_shear():
    """Like D3Q19-I (and unlike D3Q19-S), D3Q27 keeps an x-invariant axial flow
    free of transverse velocity (Sec. 4, Sec. 5.1)."""
    n = 12
    y = np.arange(n).reshape(1, n, 1)
    z = np.arange(n).reshape(n, 1, 1)
    u = np.zeros((3, n, n, 1))
    u[0] = 0.05 + 0.02 * np.sin(2 * np.pi * y / n) * np.sin(2 * np.pi * z / n)
    cfg = oracle.Config(1, n, n, tau=1.0, stencil=27)
    _, uu = oracle.run(cfg, np.ones((n, n, 1)), u, 100)
    assert np.abs(uu[1:]).max() < 1e-15


def test_d3q27_axis_permutation_equivariance():
    base = oracle.Config(5, 4, 3, collision=oracle.TRT, tau=0.65, accel=(2e-4, -1e-4, 3e-4), stencil=27)
    rng = np.random.default_rng(3)
    rho = 1 + rng.uniform(-0.02, 0.02, base.shape)
    u = rng.uniform(-0.05, 0.05, (3,) + base.shape)
    r0, u0 = oracle.run(base, rho, u, 4)
    perm = (1, 2, 0)
    n_old = (base.nx, base.ny, base.nz)
    cfg = oracle.Config(*[n_old[perm[i]] for i in range(3)], collision=oracle.TRT, tau=0.65,
                        accel=tuple(base.accel[perm[i]] for i in range(3)), stencil=27)
    np_axes = tuple(2 - perm[2 - k] for k in range(3))
    r1, u1 = oracle.run(cfg, np.transpose(rho, np_axes), np.stack([np.transpose(u[perm[i]], np_axes)
                                                                   for i in range(3)]), 4)
    assert np.abs(r1 - np.transpose(r0, np_axes)).max() < 1e-14
    for i in range(3):
        assert np.abs(u1[i] - np.transpose(u0[perm[i]], np_axes)).max() < 1e-14
