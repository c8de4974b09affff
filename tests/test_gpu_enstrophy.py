"""The FP64 enstrophy reduction (lbm_enstrophy): 1/2 <|curl u|^2> with central
differences, against its closed form for the Taylor-Green field, against the
central-difference definition evaluated in numpy on the library's own velocity
field (periodic and with half-way bounce-back walls, every storage precision),
and A/B vs AA (bitwise)."""
import math

import numpy as np
import pytest
import torch

from paper_1803_04937_gb300 import inputs
from tests._helpers import random_fields

pytestmark = pytest.mark.gpu


def _sim(nx, ny, nz, **kw):
    from paper_1803_04937_gb300.lbm import Simulation
    return Simulation(nx, ny, nz, **kw)


def _definition(u, walls):
    """1/2 mean |curl u|^2; u[3, nz, ny, nx]; ghost -u across a wall."""
    u = np.asarray(u, dtype=np.float64)

    def d(f, axis_xyz):
        ax = 2 - axis_xyz  # numpy axis of x, y, z in [z, y, x]
        up = np.roll(f, -1, ax)
        um = np.roll(f, 1, ax)
        if walls[axis_xyz]:
            n = f.shape[ax]
            sl_last = [slice(None)] * 3
            sl_last[ax] = n - 1
            sl_first = [slice(None)] * 3
            sl_first[ax] = 0
            up[tuple(sl_last)] = -f[tuple(sl_last)]
            um[tuple(sl_first)] = -f[tuple(sl_first)]
        return 0.5 * (up - um)

    ux, uy, uz = u
    wx = d(uz, 1) - d(uy, 2)
    wy = d(ux, 2) - d(uz, 0)
    wz = d(uy, 0) - d(ux, 1)
    return 0.5 * float((wx ** 2 + wy ** 2 + wz ** 2).mean())


@pytest.mark.parametrize("n", [16, 32])
def test_enstrophy_of_taylor_green_closed_form(n):
    """u = A (sin X cos Y cos Z, -cos X sin Y cos Z, 0): central differences
    replace k by sin k, and the mean of each squared product of sines and
    cosines is 1/8, so the enstrophy is (3/8) A^2 sin^2(2 pi / n)."""
    A = 0.05
    rho, u = inputs.taylor_green(n, u0=A)
    sim = _sim(n, n, n, precision="f64")
    sim.init(rho.cuda(), u.cuda())
    z = sim.enstrophy()
    want = 3 / 8 * A * A * math.sin(2 * math.pi / n) ** 2
    assert z == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("precision", ["f64", "f32", "f16s", "bf16s"])
@pytest.mark.parametrize("walls", [(False, False, False), (False, True, False), (True, True, True)])
def test_enstrophy_matches_definition(walls, precision):
    shape = (6, 10, 36)
    rho, u = random_fields(shape, seed=23)
    nz, ny, nx = shape
    sim = _sim(nx, ny, nz, precision=precision, tau=0.7, walls=walls, equilibrium="improved")
    sim.init(rho.cuda(), u.cuda() if precision == "f64" else u.float().cuda())
    sim.step(3)
    _, ug = sim.moments(torch.float64)
    z = sim.enstrophy()
    assert z == pytest.approx(_definition(ug.cpu().numpy(), walls), rel=1e-12)


def test_enstrophy_ab_equals_aa():
    shape = (5, 8, 40)
    rho, u = random_fields(shape, seed=29)
    vals = []
    for pattern in ("ab", "aa"):
        for steps in (3, 4):
            sim = _sim(40, 8, 5, precision="f32", tau=0.6, pattern=pattern)
            sim.init(rho.cuda(), u.float().cuda())
            sim.step(steps)
            vals.append(sim.enstrophy())
    assert vals[0] == vals[2] and vals[1] == vals[3]
