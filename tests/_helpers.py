"""Shared helpers of the GPU tests: run the same seeded case through the CUDA
library and through the FP64 oracle, and compare element by element."""
import numpy as np
import torch

import oracle

EQ = {"standard": oracle.STANDARD, "improved": oracle.IMPROVED}
COLL = {"srt": oracle.SRT, "trt": oracle.TRT, "mrt": oracle.MRT}


def oracle_config(nx, ny, nz, equilibrium="improved", collision="srt", tau=0.8, trt_magic=3 / 16,
                  force=(0.0, 0.0, 0.0), walls=(False, False, False), rho0_is_rho=False, stencil=19, omega_bulk=1.0,
                  omega_4=1.0, **_):
    return oracle.Config(nx, ny, nz, equilibrium=EQ[equilibrium], collision=COLL[collision], tau=tau,
                         trt_magic=trt_magic, accel=tuple(force), walls=tuple(walls), rho0_is_rho=rho0_is_rho,
                         stencil=stencil, omega_bulk=omega_bulk, omega_4=omega_4)


def random_fields(shape, seed, amp=0.05, drho=0.02):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    rho = 1 + rng.uniform(-drho, drho, (nz, ny, nx))
    u = rng.uniform(-amp, amp, (3, nz, ny, nx))
    return torch.from_numpy(rho), torch.from_numpy(u)


def gpu_to_oracle_order(stencil=19):
    """perm[q_oracle] = q_gpu with equal velocity vectors."""
    from paper_1803_04937_gb300 import lbm
    cg, wg, _ = lbm.velocity_set(stencil)
    co, wo, _ = oracle.velocity_set(stencil)
    index = {tuple(int(a) for a in v): q for q, v in enumerate(cg.tolist())}
    perm = np.array([index[tuple(int(a) for a in v)] for v in co])
    assert np.allclose(wg.numpy()[perm], wo)
    return perm


def gpu_pdfs_in_oracle_layout(sim):
    """Canonical GPU populations as f[nz, ny, nx, Q] (unshifted, float64, oracle order)."""
    g = sim.get_pdfs().double().cpu().numpy()  # [Q, nz, ny, nx], shifted
    _, w, _ = oracle.velocity_set(sim.stencil)
    perm = gpu_to_oracle_order(sim.stencil)
    f = np.moveaxis(g[perm], 0, -1) + w
    return f


def rel_maxnorm(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
