"""FP64 CPU oracle for the D3Q19 lattice Boltzmann step of Bauer & Ruede (arXiv:1803.04937).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this package.  The GPU library never does, and
this package never imports the GPU library: the two share no code.

Contents
--------
* ``lbm_oracle.c`` (wrapped here through ctypes): the lattice (Sec. 2.3), the
  standard equilibrium (Eq. 14, second order) and the improved D3Q19-I
  equilibrium (Eq. 22), the update of Eq. 15 with the Buick-Greated force and
  the velocity shift of Eq. 17, a TRT variant, an MRT variant in the monomial
  moment space with Maxwellian equilibrium moments (Sec. 3.2-3.3), periodic and half-way
  bounce-back boundaries (Sec. 5.1), and the adjoint of one step.
* ``construction.py``: the moment-matching construction of Sec. 3.1-3.2 in
  exact rational arithmetic.

Arrays: macroscopic fields are numpy arrays ``rho[nz, ny, nx]`` and
``u[3, nz, ny, nx]``; populations are ``f[nz, ny, nx, Q]`` (Q = 19, or 27 for
the D3Q27 lattice) in the oracle's own direction order (see ``velocity_set``).
"""
import ctypes
import dataclasses
import os

import numpy as np

from .build import build_oracle

Q = 19

_lib = None


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("equilibrium", ctypes.c_int), ("collision", ctypes.c_int),
        ("rho0_is_rho", ctypes.c_int), ("wall", ctypes.c_int * 3),
        ("nthreads", ctypes.c_int),
        ("tau", ctypes.c_double), ("trt_magic", ctypes.c_double),
        ("accel", ctypes.c_double * 3),
        ("stencil", ctypes.c_int),
        ("omega_bulk", ctypes.c_double), ("omega_4", ctypes.c_double),
    ]


def _load():
    global _lib
    if _lib is None:
        path = build_oracle()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        cp = ctypes.POINTER(_Cfg)
        lib.oracle_velocity_set.argtypes = [ip, dp, ip]
        lib.oracle_velocity_set_of.argtypes = [ctypes.c_int, ip, dp, ip]
        lib.oracle_velocity_set_of.restype = ctypes.c_int
        lib.oracle_equilibrium_field.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_long, dp, dp, dp]
        lib.oracle_equilibrium_field_of.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long, dp, dp,
                                                    dp]
        lib.oracle_init.argtypes = [cp, dp, dp, dp]
        lib.oracle_step.argtypes = [cp, dp, dp]
        lib.oracle_moments.argtypes = [cp, dp, dp, dp]
        lib.oracle_run.argtypes = [cp, dp, dp, ctypes.c_int, dp, dp]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_adjoint_step.argtypes = [cp, dp, dp, dp, dp]
        lib.oracle_adjoint_step.restype = ctypes.c_int
        lib.oracle_loss_velocity_l2.argtypes = [cp, dp, dp, dp, dp]
        lib.oracle_loss_velocity_l2.restype = ctypes.c_int
        lib.oracle_adjoint_init_velocity.argtypes = [cp, dp, dp, dp]
        lib.oracle_adjoint_init_velocity.restype = ctypes.c_int
        lib.oracle_domega_dtau.argtypes = [cp, dp, dp]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


STANDARD, IMPROVED = 0, 1
SRT, TRT, MRT = 0, 1, 2


@dataclasses.dataclass
class Config:
    """Parameters of one oracle run (lattice units)."""
    nx: int
    ny: int
    nz: int
    equilibrium: int = IMPROVED      # STANDARD (Eq. 14) or IMPROVED (Eq. 22)
    collision: int = SRT             # SRT (Eq. 15), TRT or MRT (Sec. 3.2-3.3)
    tau: float = 0.8
    trt_magic: float = 3.0 / 16.0
    accel: tuple = (0.0, 0.0, 0.0)   # body force a (Buick-Greated, Sec. 2.3)
    walls: tuple = (False, False, False)  # half-way bounce-back on both ends of an axis
    rho0_is_rho: bool = False        # rho0 = 1 (paper's choice) or rho0 = rho
    nthreads: int = 0                # OpenMP threads for oracle_step (0: default)
    stencil: int = 19                # 19 (D3Q19) or 27 (D3Q27, standard equilibrium)
    omega_bulk: float = 1.0          # MRT: rate of the trace of the second-order moments
    omega_4: float = 1.0             # MRT: rate of the even moments of order >= 4

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def Q(self):
        return 27 if self.stencil == 27 else 19

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    def _c(self):
        c = _Cfg()
        c.nx, c.ny, c.nz = self.nx, self.ny, self.nz
        c.equilibrium = int(self.equilibrium)
        c.collision = int(self.collision)
        c.rho0_is_rho = int(bool(self.rho0_is_rho))
        for i in range(3):
            c.wall[i] = int(bool(self.walls[i]))
            c.accel[i] = float(self.accel[i])
        c.nthreads = int(self.nthreads)
        c.tau = float(self.tau)
        c.trt_magic = float(self.trt_magic)
        c.stencil = int(self.stencil)
        c.omega_bulk = float(self.omega_bulk)
        c.omega_4 = float(self.omega_4)
        return c


def velocity_set(stencil=19):
    """Velocities c[Q,3], weights w[Q] and opposite index opp[Q] of D3Q19 (default)
    or D3Q27 (Sec. 2.3), in the oracle's own order."""
    lib = _load()
    nq = 27 if stencil == 27 else 19
    c = np.zeros((nq, 3), dtype=np.int32)
    w = np.zeros(nq)
    opp = np.zeros(nq, dtype=np.int32)
    lib.oracle_velocity_set_of(int(stencil), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                               opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return c, w, opp


def equilibrium(kind, rho, u, rho0_is_rho=False, stencil=19):
    """feq[..., Q] for rho[...] and u[3, ...]: Eq. 14 (second order) or, on
    D3Q19, Eq. 22."""
    lib = _load()
    nq = 27 if stencil == 27 else 19
    rho = _f64(rho)
    shape = rho.shape
    n = rho.size
    u = _f64(np.asarray(u).reshape(3, n))
    feq = np.zeros((n, nq))
    lib.oracle_equilibrium_field_of(int(stencil), int(kind), int(bool(rho0_is_rho)), n, _dp(rho.reshape(n)), _dp(u),
                                    _dp(feq))
    return feq.reshape(shape + (nq,))


def init(cfg: Config, rho, u):
    """f(t=0) = feq(rho, u0)."""
    lib = _load()
    rho = _f64(rho).reshape(cfg.shape)
    u = _f64(u).reshape((3,) + cfg.shape)
    f = np.zeros(cfg.shape + (cfg.Q,))
    c = cfg._c()
    lib.oracle_init(ctypes.byref(c), _dp(rho), _dp(u), _dp(f))
    return f


def step(cfg: Config, f, nsteps=1):
    """nsteps updates of Eq. 15 (collide, then push-stream)."""
    lib = _load()
    a = _f64(f).reshape(cfg.shape + (cfg.Q,)).copy()
    b = np.empty_like(a)
    c = cfg._c()
    for _ in range(nsteps):
        lib.oracle_step(ctypes.byref(c), _dp(a), _dp(b))
        a, b = b, a
    return a


def moments(cfg: Config, f):
    """rho (Eq. 16) and u (Eq. 17) of the populations f."""
    lib = _load()
    f = _f64(f).reshape(cfg.shape + (cfg.Q,))
    rho = np.zeros(cfg.shape)
    u = np.zeros((3,) + cfg.shape)
    c = cfg._c()
    lib.oracle_moments(ctypes.byref(c), _dp(f), _dp(rho), _dp(u))
    return rho, u


def run(cfg: Config, rho, u, nsteps):
    """nsteps steps from f = feq(rho, u); returns the final (rho, u)."""
    lib = _load()
    rho = _f64(rho).reshape(cfg.shape)
    u = _f64(u).reshape((3,) + cfg.shape)
    ro = np.zeros(cfg.shape)
    uo = np.zeros((3,) + cfg.shape)
    c = cfg._c()
    if lib.oracle_run(ctypes.byref(c), _dp(rho), _dp(u), int(nsteps), _dp(ro), _dp(uo)) != 0:
        raise MemoryError("oracle_run: allocation failed")
    return ro, uo


def max_threads():
    return int(_load().oracle_max_threads())


# ---------------------------------------------------------------- adjoint

def loss_velocity_l2(cfg: Config, f, u_target):
    """L = 1/2 sum_x |u(x) - u_target(x)|^2 and dL/df (rho0 = 1)."""
    lib = _load()
    f = _f64(f).reshape(cfg.shape + (cfg.Q,))
    tgt = _f64(u_target).reshape((3,) + cfg.shape)
    lam = np.zeros_like(f)
    L = ctypes.c_double(0.0)
    c = cfg._c()
    if lib.oracle_loss_velocity_l2(ctypes.byref(c), _dp(f), _dp(tgt), _dp(lam), ctypes.byref(L)) != 0:
        raise ValueError("adjoint requires rho0 = 1")
    return L.value, lam


def adjoint_step(cfg: Config, f_t, lam_next):
    """(lam_t, [dL/domega+, dL/domega-] contribution) for one step from state f_t."""
    lib = _load()
    f_t = _f64(f_t).reshape(cfg.shape + (cfg.Q,))
    lam_next = _f64(lam_next).reshape(cfg.shape + (cfg.Q,))
    lam = np.zeros_like(f_t)
    g = np.zeros(2)
    c = cfg._c()
    if lib.oracle_adjoint_step(ctypes.byref(c), _dp(f_t), _dp(lam_next), _dp(lam), _dp(g)) != 0:
        raise ValueError("adjoint requires rho0 = 1 and SRT or TRT")
    return lam, g


def adjoint_init_velocity(cfg: Config, u0, lam0):
    """dL/du0 from lam0 = dL/df(t=0), through f(0) = feq(rho, u0)."""
    lib = _load()
    u0 = _f64(u0).reshape((3,) + cfg.shape)
    lam0 = _f64(lam0).reshape(cfg.shape + (cfg.Q,))
    g = np.zeros((3,) + cfg.shape)
    c = cfg._c()
    if lib.oracle_adjoint_init_velocity(ctypes.byref(c), _dp(u0), _dp(lam0), _dp(g)) != 0:
        raise ValueError("adjoint requires rho0 = 1")
    return g


def domega_dtau(cfg: Config):
    lib = _load()
    a, b = ctypes.c_double(), ctypes.c_double()
    c = cfg._c()
    lib.oracle_domega_dtau(ctypes.byref(c), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def gradient_velocity_l2(cfg: Config, rho, u0, u_target, nsteps):
    """Loss, dL/du0 and dL/dtau of L = 1/2 sum |u(T) - u_target|^2 after nsteps.

    Plain reverse sweep over all stored states (small grids only)."""
    states = [init(cfg, rho, u0)]
    for _ in range(nsteps):
        states.append(step(cfg, states[-1]))
    L, lam = loss_velocity_l2(cfg, states[-1], u_target)
    gw = np.zeros(2)
    for t in range(nsteps - 1, -1, -1):
        lam, g = adjoint_step(cfg, states[t], lam)
        gw += g
    du0 = adjoint_init_velocity(cfg, u0, lam)
    dwp, dwm = domega_dtau(cfg)
    dtau = gw[0] * dwp + gw[1] * dwm
    return L, du0, dtau
