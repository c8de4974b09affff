"""Parity of the CUDA time step with the FP64 oracle, element by element, on
small seeded lattices that span several thread blocks and a ragged tail.

Tolerances (max-norm relative error of u, and absolute error of the
populations): FP64 storage 1e-12, FP32 storage 1e-5 after the run's steps."""
import numpy as np
import pytest
import torch

import oracle
from tests._helpers import gpu_pdfs_in_oracle_layout, oracle_config, random_fields, rel_maxnorm

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
PDF_TOL = {"f64": 1e-13, "f32": 1e-6}

CASES = [
    dict(equilibrium="improved", collision="srt", tau=0.8),
    dict(equilibrium="standard", collision="srt", tau=0.55),
    dict(equilibrium="improved", collision="trt", tau=0.6, force=(2e-4, -1e-4, 5e-5)),
    dict(equilibrium="standard", collision="trt", tau=0.9, walls=(False, True, False), force=(1e-4, 0, 0)),
    dict(equilibrium="improved", collision="srt", tau=0.7, walls=(True, False, True)),
    dict(equilibrium="improved", collision="trt", tau=0.51, walls=(True, True, True), force=(0, 1e-4, -2e-4)),
    dict(equilibrium="standard", collision="srt", tau=1.3, rho0_is_rho=True, force=(1e-4, 2e-4, 0)),
    dict(equilibrium="improved", collision="trt", tau=0.75, rho0_is_rho=True, walls=(False, True, False)),
]


def _run_gpu(shape, rho, u, steps, precision, pattern, case, cells_x=None):
    from paper_1803_04937_gb300.lbm import Simulation
    nz, ny, nx = shape
    sim = Simulation(nx, ny, nz, precision=precision, pattern=pattern, cells_x=cells_x, **case)
    sim.init(rho.cuda(), u.cuda())
    sim.step(steps)
    r, uu = sim.moments(torch.float64)
    return sim, r.cpu().numpy(), uu.cpu().numpy()


# (nx, cells per thread): odd nx with one cell per thread; even nx = 130 with two
# cells per thread spans three warps of a row, a ragged last warp and the
# cross-warp / wrap-around edge loads of the paired kernel.
MAPPINGS = [(37, 1), (130, 2)]


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("mapping", MAPPINGS)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_step_matches_oracle(case, mapping, pattern, precision):
    kw = CASES[case]
    nx, cells_x = mapping
    shape = (5, 9, nx)  # nz, ny, nx
    rho, u = random_fields(shape, seed=100 + case)
    steps = 7 if pattern == "aa" else 6  # odd count leaves AA in its odd layout
    sim, r_g, u_g = _run_gpu(shape, rho, u, steps, precision, pattern, kw, cells_x=cells_x)
    cfg = oracle_config(shape[2], shape[1], shape[0], **kw)
    f_o = oracle.step(cfg, oracle.init(cfg, rho.numpy(), u.numpy()), steps)
    r_o, u_o = oracle.moments(cfg, f_o)
    assert rel_maxnorm(u_g, u_o) < TOL[precision]
    assert np.abs(r_g - r_o).max() < TOL[precision]
    f_g = gpu_pdfs_in_oracle_layout(sim)
    assert np.abs(f_g - f_o).max() < PDF_TOL[precision]


@pytest.mark.parametrize("precision", ["f32", "f16s", "bf16s", "f64"])
@pytest.mark.parametrize("case", [0, 3, 5])
@pytest.mark.parametrize("nx", [45, 130, 388])
def test_aa_equals_ab_bitwise(nx, case, precision):
    """AA and A/B, with one, two or four cells per thread, run the same
    arithmetic per cell: identical bits after any number of steps (also a race
    check of the in-place pattern).  nx = 388 gives the four-cell 16-bit kernel
    interior warps as well as the row-end warps."""
    kw = CASES[case]
    shape = (6, 11, nx)
    rho, u = random_fields(shape, seed=7)
    for steps in (1, 4, 9):
        sa, _, _ = _run_gpu(shape, rho, u, steps, precision, "ab", kw, cells_x=1)
        sb, _, _ = _run_gpu(shape, rho, u, steps, precision, "aa", kw, cells_x=2)
        sc, _, _ = _run_gpu(shape, rho, u, steps, precision, "ab", kw, cells_x=2)
        sd, _, _ = _run_gpu(shape, rho, u, steps, precision, "ab", kw, cells_x=4)
        assert torch.equal(sa.get_pdfs(), sc.get_pdfs())
        assert torch.equal(sa.get_pdfs(), sd.get_pdfs())
        assert torch.equal(sa.get_pdfs(), sb.get_pdfs())
        ra, ua = sa.moments(torch.float32)
        rb, ub = sb.moments(torch.float32)
        assert torch.equal(ua, ub) and torch.equal(ra, rb)


# (nz, ny, nx) for the four-cell AA steps, with the block the launcher picks
# (the fewest idle lanes at a row's end): nx = 4 (one quad, its own periodic
# neighbour), 40 (a ragged warp), 64 (blocks of 32 x 4 rows, half a warp
# idle), 256 (64 x 2, whole rows), 388 (128 x 1, ragged), 600 (32 x 4, five
# blocks per row), 1000 (128 x 1, two blocks per row) and 1040 (32 x 4, nine
# blocks per row).
AA4_SHAPES = [(3, 7, 4), (4, 9, 40), (3, 8, 64), (2, 6, 256), (3, 5, 388), (2, 3, 600), (1, 2, 1000), (2, 3, 1040)]


@pytest.mark.parametrize("precision", ["f16s", "bf16s"])
@pytest.mark.parametrize("case", [0, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("shape", AA4_SHAPES)
def test_aa_four_cells_is_bitwise(shape, case, precision):
    """The four-cell AA steps (16-bit storage) against the one-cell A/B step,
    bit for bit, after even and odd step counts, over the row and block shapes
    of AA4_SHAPES; walls on x (cases 4, 5) take the shuffle kernel's scalar
    edge writes through a wall, walls on y (3, 7) and z (4, 5) the whole quad
    into the own cells."""
    kw = CASES[case]
    rho, u = random_fields(shape, seed=13)
    for steps in (1, 2, 5):
        sa, _, _ = _run_gpu(shape, rho, u, steps, precision, "ab", kw, cells_x=1)
        sb, _, _ = _run_gpu(shape, rho, u, steps, precision, "aa", kw, cells_x=4)
        assert torch.equal(sa.get_pdfs(), sb.get_pdfs())


@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("collision", ["trt", "mrt"])
@pytest.mark.parametrize("precision", ["f16s", "bf16s"])
@pytest.mark.parametrize("walls", [(False, True, False), (False, False, True), (False, True, True), (True, False, False),
                                   (True, True, True)])
@pytest.mark.parametrize("shape", [(5, 7, 40), (1, 2, 388), (2, 1, 64), (2, 2, 8), (3, 2, 4), (6, 3, 1040)])
def test_four_cell_split_rows_is_bitwise(shape, walls, precision, collision, pattern):
    """With walls on y and/or z only, the four-cell A/B step and the AA odd
    step run their interior rows through the periodic kernel and the wall rows
    through the walled one (split_rows); with walls on x as well, the A/B step
    runs the rows that touch no y/z wall through a kernel with the x-wall
    selects only.  For the TRT and the MRT collision the result is bitwise that
    of the one-cell A/B step, also on lattices of one or two rows or planes,
    which have no interior."""
    kw = dict(equilibrium="improved", collision=collision, tau=0.6, walls=walls, force=(1e-4, -2e-4, 1e-4))
    if collision == "mrt":
        kw.update(omega_bulk=1.3, omega_4=0.9)
    rho, u = random_fields(shape, seed=11)
    for steps in (1, 2, 5):
        sa, _, _ = _run_gpu(shape, rho, u, steps, precision, "ab", kw, cells_x=1)
        sb, _, _ = _run_gpu(shape, rho, u, steps, precision, pattern, kw, cells_x=4)
        assert torch.equal(sa.get_pdfs(), sb.get_pdfs()), steps


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("walls", [(False, True, False), (False, False, True), (False, True, True), (True, False, False),
                                   (True, True, True)])
@pytest.mark.parametrize("shape", [(5, 7, 37), (1, 2, 64), (2, 1, 45), (6, 3, 130)])
def test_one_cell_aa_split_rows_is_bitwise(shape, walls, precision):
    """The one-cell AA odd step on a walled lattice runs its interior rows
    through the periodic kernel (with walls on x, the kernel with the x-wall
    selects only) and the wall rows through the walled one (split_rows); after
    even and odd step counts the populations are bitwise those of the one-cell
    A/B step."""
    kw = dict(equilibrium="improved", collision="trt", tau=0.6, walls=walls, force=(1e-4, -2e-4, 1e-4))
    rho, u = random_fields(shape, seed=23)
    for steps in (1, 2, 5):
        sa, _, _ = _run_gpu(shape, rho, u, steps, precision, "ab", kw, cells_x=1)
        sb, _, _ = _run_gpu(shape, rho, u, steps, precision, "aa", kw, cells_x=1)
        assert torch.equal(sa.get_pdfs(), sb.get_pdfs()), steps


@pytest.mark.parametrize("stencil,pattern,precision", [(19, "ab", "f32"), (19, "aa", "f32"), (19, "ab", "f16s"),
                                                       (19, "aa", "bf16s"), (27, "ab", "f32"), (19, "ab", "f64")])
def test_graph_replay_is_bitwise(stencil, pattern, precision):
    """lbm_step replays captured 16-step CUDA graphs for long step counts; the
    results equal one launch per step bit for bit, across odd remainders,
    option changes (the graphs are rebuilt with the new parameters) and a
    checkpoint restore."""
    from paper_1803_04937_gb300.lbm import Simulation
    shape = (6, 10, 40)
    rho, u = random_fields(shape, seed=31)
    kw = dict(stencil=stencil, pattern=pattern, precision=precision, collision="trt", tau=0.7,
              walls=(False, True, False), force=(1e-4, 0, 0),
              equilibrium="standard" if stencil == 27 else "improved")
    sims = []
    for graphs in (True, False):
        sim = Simulation(40, 10, 6, graphs=graphs, **kw)
        sim.init(rho.cuda(), u.cuda() if precision == "f64" else u.float().cuda())
        sim.step(37)
        sim._set(_lib_opt("OPT_TAU"), 0.9)
        sim.step(16)
        sim.step(3)
        sim.step(33)
        sims.append(sim)
    assert torch.equal(sims[0].get_pdfs(), sims[1].get_pdfs())
    assert sims[0].steps_done() == sims[1].steps_done() == 89
    ck = sims[0].get_pdfs()
    sims[0].set_pdfs(ck)
    sims[0].step(20)
    sims[1].step(20)
    assert torch.equal(sims[0].get_pdfs(), sims[1].get_pdfs())


@pytest.mark.parametrize("pattern,precision", [("ab", "f32"), ("aa", "f16s")])
def test_step_captured_by_the_caller(pattern, precision):
    """A caller may capture lbm_step into its own CUDA graph (torch.cuda.graph on
    the bound stream): the library then records plain launches instead of
    replaying its own graphs.  Two replays of a captured 32-step sequence equal
    64 steps taken directly, bit for bit."""
    from paper_1803_04937_gb300.lbm import Simulation
    shape = (5, 8, 40)
    rho, u = random_fields(shape, seed=37)
    kw = dict(pattern=pattern, precision=precision, collision="trt", tau=0.7, force=(1e-4, 0, 0))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a = Simulation(40, 8, 5, stream=stream, **kw)
        a.init(rho.cuda(), u.float().cuda())
        a.step(2)  # kernels loaded before the capture
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        a.step(32)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        pa = a.get_pdfs()
    stream.synchronize()
    b = Simulation(40, 8, 5, **kw)
    b.init(rho.cuda(), u.float().cuda())
    b.step(66)
    assert torch.equal(pa, b.get_pdfs())


def _lib_opt(name):
    from paper_1803_04937_gb300 import _lib
    return getattr(_lib, name)


@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_checkpoint_restore_is_bitwise(pattern):
    from paper_1803_04937_gb300.lbm import Simulation
    shape = (4, 8, 40)
    rho, u = random_fields(shape, seed=3)
    kw = dict(collision="trt", tau=0.6, walls=(False, True, False), force=(1e-4, 0, 0))
    a = Simulation(40, 8, 4, pattern=pattern, **kw)
    a.init(rho.cuda(), u.cuda())
    a.step(5)
    ck = a.get_pdfs()
    a.step(6)
    b = Simulation(40, 8, 4, pattern=pattern, **kw)
    b.set_pdfs(ck)
    assert torch.equal(b.get_pdfs(), ck)
    b.step(6)
    assert torch.equal(a.get_pdfs(), b.get_pdfs())


def test_reductions_match_oracle_and_flag_nonfinite():
    from paper_1803_04937_gb300.lbm import Simulation
    shape = (7, 10, 33)
    rho, u = random_fields(shape, seed=9)
    kw = dict(equilibrium="improved", collision="srt", tau=0.7, force=(1e-4, -2e-4, 3e-5))
    sim = Simulation(33, 10, 7, precision="f64", **kw)
    sim.init(rho.cuda(), u.cuda())
    sim.step(5)
    red = sim.reduce()
    cfg = oracle_config(33, 10, 7, **kw)
    f = oracle.step(cfg, oracle.init(cfg, rho.numpy(), u.numpy()), 5)
    r_o, u_o = oracle.moments(cfg, f)
    c, _, _ = oracle.velocity_set()
    assert red["mass"] == pytest.approx(f.sum(), rel=1e-14)
    assert red["energy"] == pytest.approx(0.5 * (u_o ** 2).sum(), rel=1e-12)
    j = (f.reshape(-1, 19) @ c).sum(axis=0)
    assert np.allclose(red["momentum"], j, rtol=1e-12, atol=1e-14)
    assert red["umax"] == pytest.approx(np.sqrt((u_o ** 2).sum(axis=0)).max(), rel=1e-12)
    assert red["nonfinite"] == 0 and red["status"] == 0
    # deterministic
    assert sim.reduce() == red
    # a NaN planted on the host is reported, not hidden
    p = sim.get_pdfs()
    p[3, 2, 4, 5] = float("nan")
    sim.set_pdfs(p)
    bad = sim.reduce()
    assert bad["nonfinite"] == 1 and bad["status"] == 5


@pytest.mark.parametrize("precision,bound", [("f16s", 2e-3), ("bf16s", 2e-2)])
@pytest.mark.parametrize("cells_x", [1, 2])
def test_16bit_storage_error_is_bounded(cells_x, precision, bound):
    """16-bit shifted storage: velocity error against the FP64 oracle, stated."""
    shape = (8, 16, 64)
    rho, u = random_fields(shape, seed=21, amp=0.05, drho=0.0)
    kw = dict(equilibrium="improved", collision="srt", tau=0.8)
    _, _, u_g = _run_gpu(shape, rho, u, 20, precision, "ab", kw, cells_x=cells_x)
    cfg = oracle_config(64, 16, 8, **kw)
    _, u_o = oracle.run(cfg, rho.numpy(), u.numpy(), 20)
    err = rel_maxnorm(u_g, u_o)
    print("%s velocity max-norm relative error after 20 steps: %.3e" % (precision, err))
    assert err < bound


def test_tiny_and_degenerate_lattices():
    """1x1x1 (streaming is the identity), 1-cell-thick slabs in each axis, and
    walls on a 1-cell axis all agree with the oracle."""
    for shape, walls in [((1, 1, 1), (False, False, False)), ((1, 1, 7), (False, False, False)),
                         ((3, 1, 1), (False, False, True)), ((1, 5, 1), (False, True, False)),
                         ((2, 1, 3), (True, True, False)), ((2, 3, 2), (True, False, False)),
                         ((1, 1, 2), (False, False, False)), ((3, 2, 4), (True, True, True))]:
        kw = dict(collision="trt", tau=0.7, force=(1e-4, 2e-4, -1e-4), walls=walls)
        rho, u = random_fields(shape, seed=5)
        cfg = oracle_config(shape[2], shape[1], shape[0], **kw)
        _, u_o = oracle.run(cfg, rho.numpy(), u.numpy(), 5)
        for cells_x in (1, 2):
            _, _, u_g = _run_gpu(shape, rho, u, 5, "f64", "ab", kw, cells_x=cells_x)
            _, _, u_a = _run_gpu(shape, rho, u, 5, "f64", "aa", kw, cells_x=cells_x)
            assert rel_maxnorm(u_g, u_o) < 1e-12, (shape, cells_x)
            assert rel_maxnorm(u_a, u_o) < 1e-12, (shape, cells_x)


def test_zero_steps_returns_initial_fields():
    from paper_1803_04937_gb300.lbm import Simulation
    shape = (3, 4, 5)
    rho, u = random_fields(shape, seed=1)
    for pattern in ("ab", "aa"):
        sim = Simulation(5, 4, 3, precision="f64", pattern=pattern)
        sim.init(rho.cuda(), u.cuda())
        sim.step(0)
        r, uu = sim.moments()
        assert torch.allclose(r.cpu(), rho, atol=1e-15) and torch.allclose(uu.cpu(), u, atol=1e-15)


@pytest.mark.parametrize("collision,tau", [("srt", 0.55), ("srt", 0.8), ("trt", 0.6)])
@pytest.mark.parametrize("precision,tol", [("f32", 2e-6), ("f64", 1e-13)])
def test_uniform_flow_keeps_its_momentum(collision, tau, precision, tol):
    """A uniform flow is a fixed point of Eq. 15; in working precision the
    equilibrium's first moment must be exactly u, or the antisymmetric
    relaxation drifts the momentum by a constant factor every step."""
    from paper_1803_04937_gb300.lbm import Simulation
    n = 16
    U = (0.1, -0.05, 0.02)
    u = torch.zeros((3, n, n, n), dtype=torch.float64)
    for i in range(3):
        u[i] = U[i]
    sim = Simulation(n, n, n, precision=precision, collision=collision, tau=tau)
    sim.init(torch.ones((n, n, n), dtype=torch.float64).cuda(), u.cuda())
    sim.step(2000)
    _, ug = sim.moments()
    err = float((ug.cpu() - u).abs().max() / 0.1)
    print("uniform flow %s %s tau=%.2f: max|u - U|/|U_x| after 2000 steps = %.2e" % (precision, collision, tau, err))
    assert err < tol


def test_fp32_global_momentum_drift():
    """Global momentum of a random periodic flow in FP32 storage over 1000 steps
    (FP64 reduction): conserved to rounding, no systematic drift."""
    from paper_1803_04937_gb300.lbm import Simulation
    shape = (24, 24, 24)
    rho, u = random_fields(shape, seed=77, amp=0.05, drho=0.0)
    u[0] += 0.08  # mean flow
    sim = Simulation(24, 24, 24, precision="f32", collision="srt", tau=0.55)
    sim.init(rho.cuda(), u.cuda())
    j0 = np.array(sim.reduce()["momentum"])
    sim.step(1000)
    j1 = np.array(sim.reduce()["momentum"])
    drift = float(np.abs(j1 - j0).max() / np.abs(j0).max())
    print("FP32 global momentum drift over 1000 steps: %.2e" % drift)
    assert drift < 1e-6
