"""Pins of the oracle's adjoint (reverse-mode derivative of the time step) against
central finite differences of the oracle's own forward run, which shares no
code with the adjoint's explicit Jacobian."""
import numpy as np
import pytest

import oracle


def _loss(cfg, rho, u0, tgt, nsteps):
    _, u = oracle.run(cfg, rho, u0, nsteps)
    return 0.5 * ((u - tgt) ** 2).sum()


CASES = [
    dict(equilibrium=oracle.IMPROVED, collision=oracle.SRT, tau=0.7),
    dict(equilibrium=oracle.STANDARD, collision=oracle.SRT, tau=0.9),
    dict(equilibrium=oracle.IMPROVED, collision=oracle.TRT, tau=0.62, accel=(2e-4, -1e-4, 5e-5),
         walls=(False, True, False)),
    dict(equilibrium=oracle.STANDARD, collision=oracle.TRT, tau=0.8, walls=(True, False, True)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_adjoint_matches_central_differences(case):
    kw = CASES[case]
    cfg = oracle.Config(4, 5, 3, **kw)
    rng = np.random.default_rng(10 + case)
    rho = 1 + rng.uniform(-0.01, 0.01, cfg.shape)
    u0 = rng.uniform(-0.05, 0.05, (3,) + cfg.shape)
    tgt = rng.uniform(-0.05, 0.05, (3,) + cfg.shape)
    T = 6
    L, du0, dtau = oracle.gradient_velocity_l2(cfg, rho, u0, tgt, T)
    assert L == pytest.approx(_loss(cfg, rho, u0, tgt, T), rel=1e-14)
    h = 1e-6
    idx = [tuple(rng.integers(0, s) for s in (3,) + cfg.shape) for _ in range(8)]
    for i in idx:
        up, um = u0.copy(), u0.copy()
        up[i] += h
        um[i] -= h
        fd = (_loss(cfg, rho, up, tgt, T) - _loss(cfg, rho, um, tgt, T)) / (2 * h)
        assert du0[i] == pytest.approx(fd, rel=1e-6, abs=1e-10)
    ht = 1e-6
    cp = oracle.Config(4, 5, 3, **{**kw, "tau": kw["tau"] + ht})
    cm = oracle.Config(4, 5, 3, **{**kw, "tau": kw["tau"] - ht})
    fd = (_loss(cp, rho, u0, tgt, T) - _loss(cm, rho, u0, tgt, T)) / (2 * ht)
    assert dtau == pytest.approx(fd, rel=1e-6, abs=1e-10)
    assert abs(dtau) > 1e-6


def test_adjoint_rejects_compressible_mode():
    cfg = oracle.Config(2, 2, 2, rho0_is_rho=True)
    with pytest.raises(ValueError):
        oracle.loss_velocity_l2(cfg, np.zeros(cfg.shape + (19,)), np.zeros((3,) + cfg.shape))
