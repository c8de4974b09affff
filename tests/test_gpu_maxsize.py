"""Lattices near the size limit of the 32-bit cell index (nx ny nz < 2^31):
the FP16-shifted in-place AA pattern at 1280^3 = 2.097e9 cells (one 80 GB
grid) and the FP16-shifted A/B pattern at 1024 x 1024 x 1040 = 1.09e9 cells
(two 41 GB grids).  The shear wave u = (U, A sin(2 pi x / nx), 0) is invariant
in y and z, so the FP64 oracle's nx x 1 x 1 column is an exact sample of every
row: sampled rows must equal each other bit for bit and the oracle column
within the 16-bit storage error, and the FP64 mass must be conserved by the
steps (up to the rounding of their 16-bit outputs)."""
import math

import numpy as np
import pytest
import torch

import oracle
from tests._helpers import oracle_config, rel_maxnorm

pytestmark = pytest.mark.gpu


def _shear_device(nx, ny, nz, U, A):
    x = torch.arange(nx, dtype=torch.float64, device="cuda")
    u = torch.zeros((3, nz, ny, nx), dtype=torch.float32, device="cuda")
    u[0] += U
    u[1] += (A * torch.sin(2 * math.pi * x / nx)).float().view(1, 1, nx)
    return u


@pytest.mark.parametrize("shape,pattern,steps", [((1280, 1280, 1280), "aa", 7), ((1040, 1024, 1024), "ab", 6)])
def test_near_index_limit(shape, pattern, steps):
    from paper_1803_04937_gb300.lbm import Simulation
    nz, ny, nx = shape
    assert nx * ny * nz < 2 ** 31
    U, A = 0.05, 0.01
    kw = dict(equilibrium="improved", collision="srt", tau=0.8)
    sim = Simulation(nx, ny, nz, precision="f16s", pattern=pattern, **kw)
    u = _shear_device(nx, ny, nz, U, A)
    sim.init(None, u)
    del u
    torch.cuda.empty_cache()
    m0 = sim.reduce()["mass"]
    sim.step(steps)
    red = sim.reduce()
    assert red["nonfinite"] == 0
    # FP16 rounding of the initial equilibrium shifts the total mass (~1e-5 relative for this
    # flow); the steps then conserve it up to the rounding of their outputs
    print("mass: initial state %.10e (rel %+.2e from nx ny nz), after %d steps rel change %+.2e"
          % (m0, m0 / (nx * ny * nz) - 1, steps, red["mass"] / m0 - 1))
    assert abs(m0 / (nx * ny * nz) - 1) < 3e-5
    assert abs(red["mass"] / m0 - 1) < 1e-5
    _, ug = sim.moments(torch.float32)
    sim.close()
    del sim
    rng = np.random.default_rng(5)
    zs = rng.integers(0, nz, 48)
    ys = rng.integers(0, ny, 48)
    rows = [ug[:, int(z), int(y), :] for z, y in zip(zs, ys)]
    rows.append(ug[:, nz - 1, ny - 1, :])  # the last row of the lattice
    for r in rows[1:]:
        assert torch.equal(r, rows[0])
    col = rows[0].double().cpu().numpy()
    del ug, rows
    torch.cuda.empty_cache()
    cfg = oracle_config(nx, 1, 1, **kw)
    x = np.arange(nx)
    u1 = np.zeros((3, 1, 1, nx))
    u1[0] = U
    u1[1] = A * np.sin(2 * math.pi * x / nx)
    _, uo = oracle.run(cfg, np.ones((1, 1, nx)), u1, steps)
    err = rel_maxnorm(col, uo[:, 0, 0, :])
    print("%dx%dx%d FP16S %s, %d steps: rows bitwise equal, max-norm rel err vs FP64 oracle %.2e"
          % (nx, ny, nz, pattern.upper(), steps, err))
    assert err < 3e-3
