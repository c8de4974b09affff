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


def oracle_run_fp32_storage(cfg, rho, u, nsteps):
    """The oracle with FP32 storage: every oracle step (FP64 arithmetic) is
    followed by rounding the shifted populations f_q - w_q to float32, which is
    what FP32 storage does to the state between steps.  Separates the error
    that storage alone causes from the error of the GPU's FP32 arithmetic.
    Returns the final (rho, u)."""
    _, w, _ = oracle.velocity_set(cfg.stencil)
    f = oracle.init(cfg, rho, u)
    f = w + (f - w).astype(np.float32).astype(np.float64)
    for _ in range(nsteps):
        f = oracle.step(cfg, f, 1)
        f = w + (f - w).astype(np.float32).astype(np.float64)
    return oracle.moments(cfg, f)


# ---------------------------------------------------------------- linear stability of uniform flow

def _d3q19_velocities():
    """D3Q19 velocities and weights enumerated here (rest, faces, edges; Sec. 2.3)."""
    c = [(0, 0, 0)]
    c += [v for v in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))]
    c += [(a, b, 0) for a in (1, -1) for b in (1, -1)]
    c += [(a, 0, b) for a in (1, -1) for b in (1, -1)]
    c += [(0, a, b) for a in (1, -1) for b in (1, -1)]
    c = np.array(c, dtype=np.float64)
    n2 = (c * c).sum(axis=1)
    w = np.where(n2 == 0, 1 / 3, np.where(n2 == 1, 1 / 18, 1 / 36))
    return c, w


def srt_collision_jacobian(U, improved, tau):
    """d f* / d f of one SRT collision (Eq. 15, no force, rho0 = 1) at the
    equilibrium of rho = 1, u = U, written from the derivatives of Eq. 14
    (second order) and of the D3Q19-I corrections of Eq. 22 (rest + u^2/6,
    face along a - (u^2 - u_a^2)/12, edge normal to c + u_c^2/24).  Returns
    (J, c) with c the velocities in this function's own order."""
    c, w = _d3q19_velocities()
    U = np.asarray(U, dtype=np.float64)
    q = len(w)
    dfeq_drho = w.copy()
    dfeq_du = np.zeros((q, 3))
    for i in range(q):
        cu = c[i] @ U
        dfeq_du[i] = w[i] * (3 * c[i] + 9 * cu * c[i] - 3 * U)
        if improved:
            n2 = int(c[i] @ c[i])
            if n2 == 0:
                dfeq_du[i] += U / 3
            elif n2 == 1:
                e = np.abs(c[i])
                dfeq_du[i] -= (U - U * e) / 6
            else:
                e = 1 - np.abs(c[i])  # the axis normal to the edge's plane
                dfeq_du[i] += U * e / 12
    E = np.outer(dfeq_drho, np.ones(q)) + dfeq_du @ c.T  # rho = sum f, u = sum c f
    omega = 1 / tau
    return np.eye(q) - omega * (np.eye(q) - E), c


def srt_max_amplification(U, improved, tau, n):
    """Largest |eigenvalue| of the linearised stream + collide step over the
    wave vectors of a periodic n^3 lattice (von Neumann analysis of the
    uniform flow U)."""
    J, c = srt_collision_jacobian(U, improved, tau)
    ks = 2 * np.pi * np.arange(n) / n
    kk = np.stack(np.meshgrid(ks, ks, ks, indexing="ij"), axis=-1).reshape(-1, 3)
    ph = np.exp(-1j * (kk @ c.T))  # [nk, Q]
    G = ph[:, :, None] * J[None, :, :]
    return float(np.abs(np.linalg.eigvals(G)).max())


# ---------------------------------------------------------------- one step of sampled cells at full size

def _storage_spacing(v, precision):
    """Spacing of the storage type at |v| (float64 array)."""
    a = np.abs(v)
    if precision == "f32":
        return np.spacing(a.astype(np.float32)).astype(np.float64)
    if precision == "f16s":
        return np.spacing(a.astype(np.float16)).astype(np.float64)
    if precision == "bf16s":  # 8 significant bits: 2^16 times the float32 spacing
        return np.spacing(a.astype(np.float32)).astype(np.float64) * 65536.0
    return np.spacing(a)


def _axis_patch(c, n, walled):
    """Rows of a patch around coordinate c along an axis of n cells, the index
    of c in it, and whether the patch is walled along that axis: next to a wall
    the two cells at the wall (walls at both patch ends; only the one the centre
    touches matters), else the three cells c - 1, c, c + 1 (periodic wrap)."""
    if walled and n == 1:
        return [c], 0, True
    if walled and c == 0:
        return [0, 1], 0, True
    if walled and c == n - 1:
        return [n - 2, n - 1], 1, True
    return [(c - 1) % n, c, (c + 1) % n], 1, False


def one_step_sampled_errors(sim, pts, kw, precision, slack):
    """Runs one GPU step of `sim` (D3Q19 or D3Q27, no walls on x) and compares it, at the
    cells pts[S] = (z, y, x), with the FP64 oracle's step of each cell's
    neighbourhood taken from the GPU's state before the step: the centre of a
    patch pulls only from the patch, so the oracle's step of the patch is the
    exact step of that cell.  Returns (largest difference in units of half an
    ulp of the stored shifted value plus `slack`, largest absolute difference)."""
    assert not kw.get("walls", (False, False, False))[0]
    walls = kw.get("walls", (False, False, False))
    nz, ny, nx = sim.shape
    perm = gpu_to_oracle_order(sim.stencil)
    _, w, _ = oracle.velocity_set(sim.stencil)
    f0 = sim.get_pdfs()
    patches = []
    for z, y, x in pts:
        zr, zc, zw = _axis_patch(int(z), nz, walls[2])
        yr, yc, yw = _axis_patch(int(y), ny, walls[1])
        xr, xc, _ = _axis_patch(int(x), nx, False)
        idx = [torch.tensor(r, device=f0.device) for r in (zr, yr, xr)]
        p = f0[:, idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]].double().cpu().numpy()
        patches.append((p, (zc, yc, xc), (zw, yw)))
    del f0
    torch.cuda.empty_cache()
    sim.step(1)
    f1 = sim.get_pdfs()
    t = [torch.tensor([int(q[i]) for q in pts], device=f1.device) for i in range(3)]
    got = f1[:, t[0], t[1], t[2]].double().cpu().numpy().T  # [S, Q] shifted, GPU order
    del f1
    torch.cuda.empty_cache()
    worst = worst_abs = 0.0
    for s, (p, (zc, yc, xc), (zw, yw)) in enumerate(patches):
        pz, py, px = p.shape[1:]
        cfg = oracle_config(px, py, pz, **dict(kw, walls=(False, yw, zw), stencil=sim.stencil))
        fo = np.moveaxis(p[perm], 0, -1) + w
        want = oracle.step(cfg, fo, 1)[zc, yc, xc] - w
        g = got[s][perm]
        d = np.abs(g - want)
        unit = 0.5 * _storage_spacing(np.maximum(np.abs(g), np.abs(want)), precision) + slack
        worst = max(worst, float((d / unit).max()))
        worst_abs = max(worst_abs, float(d.max()))
    return worst, worst_abs
