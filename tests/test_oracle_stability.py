"""Linear (von Neumann) stability of a uniform flow under SRT close to
tau = 1/2, for the standard (Eq. 14) and the improved (Eq. 22) equilibrium.

The paper reports that its plain BGK (SRT) nozzle run at a relaxation rate near
2 became unstable and switched to an entropically stabilised MRT (Sec. 5.2);
the decaying-turbulence workload runs SRT at tau = 0.51 (omega = 1.96), where
D3Q19-I blows up on the GPU and D3Q19-S does not.  These tests tie that to the
schemes themselves: the linearised step about a uniform flow U has growing
modes for D3Q19-I at |U| = 0.1 (largest growth factor about 1.0155 per step on
a 16^3 lattice, grid-scale wave vectors) while D3Q19-S has none, and the
oracle's own time step shows the predicted growth rate.

The Jacobian comes from a separate derivation (tests/_helpers.py, derivatives
of Eq. 14 and Eq. 22); it is pinned to the oracle's collision by central
differences, so a dropped or mis-signed term on either side fails."""
import numpy as np
import pytest

import oracle
from tests._helpers import srt_collision_jacobian, srt_max_amplification


def _oracle_collision_jacobian(eq, tau, U, h=1e-6, collision=oracle.SRT, trt_magic=3 / 16):
    """Central differences of one oracle step on a 1x1x1 periodic lattice
    (streaming is the identity there, so the step is one collision)."""
    cfg = oracle.Config(1, 1, 1, equilibrium=eq, collision=collision, tau=tau, trt_magic=trt_magic)
    feq = oracle.equilibrium(eq, np.ones((1, 1, 1)), np.asarray(U, dtype=np.float64).reshape(3, 1, 1, 1))
    feq = feq.reshape(19)
    J = np.zeros((19, 19))
    for p in range(19):
        fp, fm = feq.copy(), feq.copy()
        fp[p] += h
        fm[p] -= h
        J[:, p] = (oracle.step(cfg, fp.reshape(1, 1, 1, 19)).reshape(19)
                   - oracle.step(cfg, fm.reshape(1, 1, 1, 19)).reshape(19)) / (2 * h)
    c, _, _ = oracle.velocity_set()
    return J, c


@pytest.mark.parametrize("eq", [oracle.STANDARD, oracle.IMPROVED])
def test_collision_jacobian_matches_the_oracle(eq):
    U = (0.1, -0.05, 0.03)
    J, c = srt_collision_jacobian(U, eq == oracle.IMPROVED, 0.51)
    Jo, co = _oracle_collision_jacobian(eq, 0.51, U)
    index = {tuple(int(a) for a in v): i for i, v in enumerate(c)}
    perm = np.array([index[tuple(int(a) for a in v)] for v in co])  # oracle q -> helper q
    Jh = J[np.ix_(perm, perm)]
    assert np.abs(Jh - Jo).max() < 1e-8
    # the two equilibria's Jacobians differ (the D3Q19-I corrections are not lost)
    J_other, _ = srt_collision_jacobian(U, eq != oracle.IMPROVED, 0.51)
    assert np.abs(J_other[np.ix_(perm, perm)] - Jo).max() > 1e-3


def test_uniform_flow_growth_factors_at_tau_051():
    """16^3 wave vectors, tau = 0.51: at rest both schemes are neutral; at
    |U| = 0.1 along x D3Q19-I has a growing mode and D3Q19-S has none."""
    for improved in (False, True):
        assert srt_max_amplification((0, 0, 0), improved, 0.51, 16) <= 1 + 1e-12
    assert srt_max_amplification((0.1, 0, 0), False, 0.51, 16) <= 1 + 1e-12
    g_i = srt_max_amplification((0.1, 0, 0), True, 0.51, 16)
    assert 1.010 < g_i < 1.020
    # a viscous tau keeps both stable at the same speed
    assert srt_max_amplification((0.1, 0, 0), True, 0.8, 16) <= 1 + 1e-12


def test_oracle_step_grows_at_the_predicted_rate():
    """The oracle's time step on a periodic 16^3 lattice, uniform U = 0.1 e_x
    plus a seeded 1e-9 velocity perturbation, tau = 0.51, 800 steps: under
    D3Q19-I the perturbation grows at the largest linear growth factor (about
    e^6 over the last 400 steps), under D3Q19-S it does not grow."""
    n, tau = 16, 0.51
    rng = np.random.default_rng(5)
    u = np.zeros((3, n, n, n))
    u[0] = 0.1
    u += 1e-9 * rng.standard_normal(u.shape)
    rho = np.ones((n, n, n))
    amp = {}
    for eq in (oracle.STANDARD, oracle.IMPROVED):
        cfg = oracle.Config(n, n, n, equilibrium=eq, collision=oracle.SRT, tau=tau)
        f = oracle.init(cfg, rho, u)
        a = []
        for t in range(0, 801, 200):
            if t:
                f = oracle.step(cfg, f, 200)
            _, uo = oracle.moments(cfg, f)
            uo[0] -= 0.1
            a.append(np.abs(uo).max())
        amp[eq] = a
    g = srt_max_amplification((0.1, 0, 0), True, tau, n)
    # after the other modes have decayed (steps 400 -> 800) the largest one sets the rate
    rate = (np.log(amp[oracle.IMPROVED][4]) - np.log(amp[oracle.IMPROVED][2])) / 400
    assert rate == pytest.approx(np.log(g), rel=0.03)
    assert amp[oracle.STANDARD][4] <= amp[oracle.STANDARD][0]


def _max_amplification(J, c, n):
    ks = 2 * np.pi * np.arange(n) / n
    kk = np.stack(np.meshgrid(ks, ks, ks, indexing="ij"), axis=-1).reshape(-1, 3)
    G = np.exp(-1j * (kk @ c.T.astype(np.float64)))[:, :, None] * J[None]
    return float(np.abs(np.linalg.eigvals(G)).max())


@pytest.mark.parametrize("magic", [1e-4, 3 / 16])
def test_trt_does_not_stabilise_the_improved_equilibrium_at_tau_051(magic):
    """TRT (Sec. 3.3) at tau = 0.51 with a small or the usual magic parameter,
    linearised from the oracle's own collision: D3Q19-I still has a growing
    mode at |U| = 0.1 along x, D3Q19-S none."""
    for eq, grows in ((oracle.IMPROVED, True), (oracle.STANDARD, False)):
        J, c = _oracle_collision_jacobian(eq, 0.51, (0.1, 0.0, 0.0), collision=oracle.TRT, trt_magic=magic)
        g = _max_amplification(J, c, 16)
        if grows:
            assert g > 1.01
        else:
            assert g < 1 + 1e-6
