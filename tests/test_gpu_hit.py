"""Decaying homogeneous isotropic turbulence: periodic 768^3, tau = 0.51, SRT,
solenoidal initial field with E(k) ~ k^4 exp(-2 (k/4)^2), u_rms = 0.04
(seed 4), 2000 steps, FP16-shifted vs FP32 storage, both equilibria.  The flow
is chaotic, so the 768^3 runs are not compared point by point with the oracle
(parity unpinned at this size); instead the same seed at 192^3 runs in FP64 on
the GPU, which is pinned to the CPU oracle for the first steps, and the 16- and
32-bit storage runs are compared with it (energy and enstrophy series)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1803_04937_gb300 import inputs
from tests._helpers import oracle_config, rel_maxnorm

pytestmark = pytest.mark.gpu


def _series(n, precision, equilibrium, steps, every, pattern="aa"):
    from paper_1803_04937_gb300.lbm import Simulation
    sim = Simulation(n, n, n, equilibrium=equilibrium, collision="srt", tau=0.51, precision=precision,
                     pattern=pattern)
    rho, u = inputs.hit_spectrum(n, n, n, u_rms=0.04, seed=4, device="cuda")
    sim.init(None, u if precision == "f64" else u.float())
    del rho, u
    E, Z = [], []
    for t in range(0, steps + 1, every):
        if t:
            sim.step(every)
        red = sim.reduce()
        if red["nonfinite"]:
            E.append(float("nan"))
            Z.append(float("nan"))
            break
        E.append(red["energy"] / sim.ncell)
        Z.append(sim.enstrophy())
    sim.close()
    return np.array(E), np.array(Z)


def test_hit_192_fp64_gpu_matches_oracle():
    n, steps = 192, 40
    rho, u = inputs.hit_spectrum(n, n, n, u_rms=0.04, seed=4)
    from paper_1803_04937_gb300.lbm import Simulation
    for equilibrium in ("standard", "improved"):
        kw = dict(equilibrium=equilibrium, collision="srt", tau=0.51)
        sim = Simulation(n, n, n, precision="f64", **kw)
        sim.init(None, u.cuda())
        sim.step(steps)
        _, ug = sim.moments()
        cfg = oracle_config(n, n, n, **kw)
        _, uo = oracle.run(cfg, rho.numpy(), u.numpy(), steps)
        err = rel_maxnorm(ug.cpu().numpy(), uo)
        print("HIT 192^3 FP64 GPU vs oracle after %d steps (%s): %.2e" % (steps, equilibrium, err))
        assert err < 1e-12


def test_hit_storage_precision_against_fp64():
    """192^3, same seed: FP32 and FP16-shifted storage against the FP64 GPU run
    (energy and enstrophy series, 2000 steps)."""
    n, steps, every = 192, 2000, 100
    for equilibrium in ("standard", "improved"):
        E64, Z64 = _series(n, "f64", equilibrium, steps, every)
        for precision in ("f32", "f16s"):
            E, Z = _series(n, precision, equilibrium, steps, every)
            m = min(len(E), len(E64))
            de = np.nanmax(np.abs(E[:m] / E64[:m] - 1))
            dz = np.nanmax(np.abs(Z[:m] / Z64[:m] - 1))
            print("HIT 192^3 %s %s vs FP64: max rel dev energy %.2e, enstrophy %.2e (E0 %.3e, E_end %.3e)"
                  % (equilibrium, precision, de, dz, E64[0], E64[-1]))
            if precision == "f32":
                assert de < 1e-3 and dz < 1e-2


def test_hit_768_series():
    """The full 768^3 runs (AA pattern): FP16-shifted vs FP32 energy and
    enstrophy series for both equilibria; reports a blow-up if one happens."""
    n, steps, every = 768, 2000, 250
    res = {}
    for equilibrium in ("standard", "improved"):
        for precision in ("f32", "f16s"):
            E, Z = _series(n, precision, equilibrium, steps, every)
            res[(equilibrium, precision)] = (E, Z)
            print("HIT 768^3 %s %s: E(t) %s" % (equilibrium, precision, np.array2string(E, precision=4)))
            print("HIT 768^3 %s %s: Z(t) %s" % (equilibrium, precision, np.array2string(Z, precision=4)))
    for equilibrium in ("standard", "improved"):
        E32, Z32 = res[(equilibrium, "f32")]
        E16, Z16 = res[(equilibrium, "f16s")]
        m = min(len(E32), len(E16))
        print("HIT 768^3 %s FP16S vs FP32: max rel dev energy %.2e, enstrophy %.2e"
              % (equilibrium, np.nanmax(np.abs(E16[:m] / E32[:m] - 1)), np.nanmax(np.abs(Z16[:m] / Z32[:m] - 1))))
        assert np.isfinite(E32[0]) and E32[0] > 0
