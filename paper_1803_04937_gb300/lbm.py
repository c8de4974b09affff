"""Python front end of the D3Q19 library: a ``Simulation`` owns torch-allocated
device buffers and drives the C ABI (include/lbm.h) through ctypes.

Every computation runs in the CUDA kernels of ``liblbm_gb300.so``; this module
only allocates memory, marshals pointers and checks status codes.
"""
import ctypes

import torch

from . import _lib
from ._lib import check

_PRECISION = {"f64": _lib.F64, "f32": _lib.F32, "f16s": _lib.F16S, "bf16s": _lib.BF16S}
_STORAGE_DTYPE = {_lib.F64: torch.float64, _lib.F32: torch.float32, _lib.F16S: torch.float16,
                  _lib.BF16S: torch.bfloat16}
_EQ = {"standard": _lib.EQ_STANDARD, "improved": _lib.EQ_IMPROVED}
_COLL = {"srt": _lib.SRT, "trt": _lib.TRT, "mrt": _lib.MRT}
_PATTERN = {"ab": _lib.PATTERN_AB, "aa": _lib.PATTERN_AA}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _field_dtype(t):
    if t.dtype == torch.float64:
        return _lib.DTYPE_F64
    if t.dtype == torch.float32:
        return _lib.DTYPE_F32
    raise TypeError("macroscopic fields must be float64 or float32, got %s" % t.dtype)


def velocity_set(stencil=19):
    """(c[Q,3], w[Q], opp[Q]) in the library's D3Q19 (default) or D3Q27 order."""
    lib = _lib.load()
    nq = int(stencil)
    c = (ctypes.c_int * (3 * nq))()
    w = (ctypes.c_double * nq)()
    o = (ctypes.c_int * nq)()
    check(lib.lbm_velocity_set_of(nq, c, w, o))
    return (torch.tensor(list(c), dtype=torch.int64).view(nq, 3), torch.tensor(list(w), dtype=torch.float64),
            torch.tensor(list(o), dtype=torch.int64))


class Simulation:
    """One D3Q19 lattice on one GPU.

    Parameters mirror ``lbm_create`` / ``lbm_set_option``: equilibrium
    ("standard" = Eq. 14, "improved" = Eq. 22), collision ("srt" | "trt" |
    "mrt"), tau, storage precision ("f64" | "f32" | "f16s" | "bf16s"), TRT magic
    parameter (also the odd-moment rate of MRT), the MRT bulk and fourth-order
    rates ``omega_bulk`` and ``omega_4``,
    body force a, half-way bounce-back walls per axis, rho0 mode and
    propagation pattern ("ab" | "aa").  ``stencil=27`` selects the D3Q27
    comparison lattice (A/B pattern, standard equilibrium).  Work is enqueued on
    ``stream`` (default: torch's current stream on ``device``).
    """

    def __init__(self, nx, ny, nz, equilibrium="improved", collision="srt", tau=0.8, precision="f32",
                 trt_magic=3.0 / 16.0, force=(0.0, 0.0, 0.0), walls=(False, False, False), rho0_is_rho=False,
                 pattern="ab", device="cuda", stream=None, block=None, cells_x=None, stencil=19, omega_bulk=1.0,
                 omega_4=1.0, graphs=None):
        self._lib = lib = _lib.load()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("the D3Q19 library runs on CUDA devices only")
        self.precision = _PRECISION[precision]
        self.storage_dtype = _STORAGE_DTYPE[self.precision]
        h = ctypes.c_void_p()
        self.stencil = int(stencil)
        check(lib.lbm_create(self.nx, self.ny, self.nz, self.stencil, _EQ[equilibrium], _COLL[collision],
                             float(tau), self.precision, ctypes.byref(h)))
        self._h = h
        self._set(_lib.OPT_TRT_MAGIC, trt_magic)
        if collision == "mrt":
            self._set(_lib.OPT_MRT_OMEGA_BULK, omega_bulk)
            self._set(_lib.OPT_MRT_OMEGA_4, omega_4)
        for i in range(3):
            self._set(_lib.OPT_FORCE_X + i, force[i])
            self._set(_lib.OPT_WALLS_X + i, 1.0 if walls[i] else 0.0)
        self._set(_lib.OPT_RHO0_MODE, 1.0 if rho0_is_rho else 0.0)
        self._set(_lib.OPT_PATTERN, _PATTERN[pattern])
        if block is not None:
            self._set(_lib.OPT_BLOCK_Y, 1)  # keep bx * by valid while changing bx
            self._set(_lib.OPT_BLOCK_X, block[0])
            self._set(_lib.OPT_BLOCK_Y, block[1])
        if cells_x is not None:
            self._set(_lib.OPT_CELLS_X, cells_x)
        if graphs is not None:
            self._set(_lib.OPT_GRAPHS, 1.0 if graphs else 0.0)
        self.pattern = pattern
        pdf_bytes = ctypes.c_size_t()
        ngrids = ctypes.c_int()
        scratch_bytes = ctypes.c_size_t()
        check(lib.lbm_required_bytes(h, ctypes.byref(pdf_bytes), ctypes.byref(ngrids), ctypes.byref(scratch_bytes)), h)
        self.pdf_bytes = pdf_bytes.value
        shape = (self.stencil, self.nz, self.ny, self.nx)
        self.grids = [torch.empty(shape, dtype=self.storage_dtype, device=self.device) for _ in range(ngrids.value)]
        self.scratch = torch.zeros(scratch_bytes.value // 8, dtype=torch.float64, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._bind(self.grids[0], self.grids[1] if len(self.grids) > 1 else None)

    # -- low level ---------------------------------------------------------
    def _set(self, key, value):
        check(self._lib.lbm_set_option(self._h, key, float(value)), self._h)

    def _bind(self, a, b=None):
        check(self._lib.lbm_bind(self._h, _ptr(a), _ptr(b), _ptr(self.scratch),
                                 ctypes.c_void_p(self.stream.cuda_stream)), self._h)

    def option(self, key):
        v = ctypes.c_double()
        check(self._lib.lbm_get_option(self._h, key, ctypes.byref(v)), self._h)
        return v.value

    @property
    def handle(self):
        return self._h

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    # -- state -------------------------------------------------------------
    def init(self, rho, u):
        """f = feq(rho, u) (Eq. 14 or Eq. 22); rho[nz,ny,nx] (or None) and u[3,nz,ny,nx]."""
        u = u.to(self.device).contiguous()
        dt = _field_dtype(u)
        if rho is not None:
            rho = rho.to(device=self.device, dtype=u.dtype).contiguous()
        self._keep = (rho, u)  # kept alive until the kernel has run
        check(self._lib.lbm_init(self._h, _ptr(rho), _ptr(u), dt), self._h)

    def step(self, n=1):
        check(self._lib.lbm_step(self._h, int(n)), self._h)

    def moments(self, dtype=torch.float64):
        """(rho[nz,ny,nx], u[3,nz,ny,nx]) of the current state (Eq. 16, Eq. 17)."""
        rho = torch.empty(self.shape, dtype=dtype, device=self.device)
        u = torch.empty((3,) + self.shape, dtype=dtype, device=self.device)
        self.moments_into(rho, u)
        return rho, u

    def moments_into(self, rho, u):
        dt = _field_dtype(u if u is not None else rho)
        check(self._lib.lbm_moments(self._h, _ptr(rho), _ptr(u), dt), self._h)

    def reduce(self):
        """FP64 global mass, energy, momentum, max |u| and non-finite count (synchronises)."""
        out = (ctypes.c_double * _lib.RED_COUNT)()
        s = self._lib.lbm_reduce(self._h, out)
        if s not in (_lib.LBM_OK, _lib.LBM_ENONFINITE):
            check(s, self._h)
        return {"mass": out[0], "energy": out[1], "momentum": (out[2], out[3], out[4]), "umax": out[5],
                "nonfinite": int(out[6]), "status": s}

    def enstrophy(self):
        """FP64 enstrophy 1/2 <|curl u|^2> of the current state (central differences; synchronises)."""
        out = ctypes.c_double()
        check(self._lib.lbm_enstrophy(self._h, ctypes.byref(out)), self._h)
        return out.value

    def steps_done(self):
        t = ctypes.c_longlong()
        check(self._lib.lbm_steps_done(self._h, ctypes.byref(t)), self._h)
        return t.value

    def get_pdfs(self):
        """Canonical copy f_q - w_q as [Q, nz, ny, nx] in storage precision."""
        out = torch.empty((self.stencil,) + self.shape, dtype=self.storage_dtype, device=self.device)
        check(self._lib.lbm_get_pdfs(self._h, _ptr(out)), self._h)
        return out

    def set_pdfs(self, pdfs):
        pdfs = pdfs.to(device=self.device, dtype=self.storage_dtype).contiguous()
        self._keep = (pdfs,)
        check(self._lib.lbm_set_pdfs(self._h, _ptr(pdfs)), self._h)

    # -- end to end from host memory -----------------------------------------
    def run_host(self, rho_host, u_host, nsteps, out=None):
        """End-to-end call from host memory: lbm_init reads rho, u straight from
        the pinned host tensors (the kernel reaches them through their mapped
        device address, no staging copy), nsteps steps run, and lbm_moments
        writes rho, u straight into ``out`` (pinned host tensors, allocated if
        None).  Synchronises the stream; returns (rho, u)."""
        for t in (rho_host, u_host) + (tuple(out) if out is not None else ()):
            if t is not None and not (t.device.type == "cpu" and t.is_pinned() and t.is_contiguous()):
                raise ValueError("run_host takes contiguous pinned host tensors")
        dt = _field_dtype(u_host)
        if out is None:
            out = (torch.empty(self.shape, dtype=u_host.dtype, pin_memory=True),
                   torch.empty((3,) + self.shape, dtype=u_host.dtype, pin_memory=True))
        check(self._lib.lbm_init(self._h, _ptr(rho_host), _ptr(u_host), dt), self._h)
        check(self._lib.lbm_step(self._h, int(nsteps)), self._h)
        check(self._lib.lbm_moments(self._h, _ptr(out[0]), _ptr(out[1]), dt), self._h)
        self.stream.synchronize()
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lbm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
