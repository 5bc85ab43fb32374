"""GB300-native homogenized lattice BGK (HBGK) library: Python binding.

The compute runs in libhlbm.so (hand-written CUDA for sm_103a behind the C ABI
declared in include/hlbm.h). This module only marshals arguments: every
``hlbm_*`` function here has the name and meaning of the C call it wraps,
takes device buffers as torch CUDA tensors (or raw integer pointers) and host
buffers as numpy arrays, and turns a negative status into ``HlbmError``.
PyTorch supplies device memory and the current CUDA stream.

There is no CPU fallback: if the shared library is missing or fails to load,
every call raises.

Method: BGK relaxation toward the homogenized Maxwellian evaluated at the
porosity-scaled velocity varpi*u (Simonis et al., arXiv:2310.14746, Part I,
Sec. 3.2, eqs. porousVeloMaxwellian, "d definition", HBGKBE).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhlbm.so")

# ---- constants (include/hlbm.h) -------------------------------------------
HLBM_OK = 0
HLBM_ERR_INVALID_ARG = -1
HLBM_ERR_OOM = -2
HLBM_ERR_CUDA = -3
HLBM_ERR_NOT_CONVERGED = -4
HLBM_ERR_TIMEOUT = -5
HLBM_ERR_BUSY = -6
HLBM_ERR_IO = -7
HLBM_ERR_STATE = -8
HLBM_ERR_CANCELLED = -9
HLBM_ERR_SCRATCH_LIMIT = -10

HLBM_D2Q9 = 9
HLBM_D3Q19 = 19
HLBM_F64 = 0
HLBM_F32 = 1
HLBM_F16DEV = 2
HLBM_BF16DEV = 3
HLBM_TWO_LATTICE = 0
HLBM_AA = 1
HLBM_PERIODIC = 0
HLBM_HALFWAY_BOUNCE_BACK = 1
HLBM_HOMOG_SHIFT = 0
HLBM_HOMOG_DRAG = 1
HLBM_STEP_AUTO = 0
HLBM_STEP_PER_CELL = 1

STAT_KEYS = ("mass", "mom_x", "mom_y", "mom_z", "plane_flux", "k_app", "max_du", "max_u")
STORAGE_BYTES = {HLBM_F64: 8, HLBM_F32: 4, HLBM_F16DEV: 2, HLBM_BF16DEV: 2}
STORAGE_NAMES = {HLBM_F64: "f64", HLBM_F32: "f32", HLBM_F16DEV: "f16dev", HLBM_BF16DEV: "bf16dev"}


class HlbmError(RuntimeError):
    def __init__(self, status, call):
        self.status = status
        msg = "%s failed: %s (%d)" % (call, _strerror(status), status)
        if status == HLBM_ERR_CUDA or status == HLBM_ERR_OOM:
            msg += " [%s]" % _lib().hlbm_last_cuda_error().decode()
        super().__init__(msg)


class hlbm_stats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3),
                ("plane_flux", ctypes.c_double), ("k_app", ctypes.c_double),
                ("max_du", ctypes.c_double), ("max_u", ctypes.c_double),
                ("step", ctypes.c_longlong)]

    def as_dict(self):
        return {"mass": self.mass, "mom_x": self.momentum[0], "mom_y": self.momentum[1],
                "mom_z": self.momentum[2], "plane_flux": self.plane_flux, "k_app": self.k_app,
                "max_du": self.max_du, "max_u": self.max_u, "step": int(self.step)}


class hlbm_request(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("tau", ctypes.c_double), ("F", ctypes.c_double * 3),
                ("varpi", ctypes.c_void_p), ("tol", ctypes.c_double), ("max_steps", ctypes.c_longlong),
                ("u_out", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


class hlbm_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("steps", ctypes.c_longlong), ("k_app", ctypes.c_double), ("max_du", ctypes.c_double),
                ("max_u", ctypes.c_double), ("mass", ctypes.c_double), ("plane_flux", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_finish", ctypes.c_double),
                ("steps_low", ctypes.c_longlong), ("final_storage", ctypes.c_int)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k == "F" else getattr(self, k)) for k, _ in self._fields_}


class hlbm_server_stats(ctypes.Structure):
    _fields_ = [("active", ctypes.c_int), ("waiting", ctypes.c_int), ("done_unpolled", ctypes.c_int),
                ("mem_used", ctypes.c_size_t), ("mem_budget", ctypes.c_size_t),
                ("lattice_updates", ctypes.c_longlong), ("rounds", ctypes.c_longlong),
                ("elapsed_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_L = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double

# name -> (restype, argtypes); every symbol include/hlbm.h declares
SIGNATURES = {
    "hlbm_create": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _i, _i, _i, _vp]),
    "hlbm_destroy": (None, [_vp]),
    "hlbm_release_scratch": (_i, [_vp]),
    "hlbm_set_stream": (_i, [_vp, _vp]),
    "hlbm_set_relaxation": (_i, [_vp, _d]),
    "hlbm_set_porosity": (_i, [_vp, _vp, _i]),
    "hlbm_set_porosity_tensor": (_i, [_vp, _vp, _i]),
    "hlbm_set_solid_mask": (_i, [_vp, _vp, _i]),
    "hlbm_porosity_from_permeability": (_i, [_vp, _d, _d, _vp, ctypes.c_size_t]),
    "hlbm_set_force": (_i, [_vp, _d, _d, _d]),
    "hlbm_set_boundary": (_i, [_vp, _i, _i]),
    "hlbm_set_storage_scale": (_i, [_vp, _d]),
    "hlbm_set_homogenization": (_i, [_vp, _i]),
    "hlbm_set_step_kernel": (_i, [_vp, _i]),
    "hlbm_init_equilibrium": (_i, [_vp, _d, _d, _d, _d]),
    "hlbm_set_populations": (_i, [_vp, _vp, _i]),
    "hlbm_get_populations": (_i, [_vp, _vp, _i]),
    "hlbm_step": (_i, [_vp, ctypes.c_long]),
    "hlbm_get_step": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "hlbm_moments": (_i, [_vp, _vp, _vp, _i]),
    "hlbm_moments_f64": (_i, [_vp, _vp, _vp, _i]),
    "hlbm_reduce": (_i, [_vp, ctypes.POINTER(hlbm_stats)]),
    "hlbm_adjoint_flux_grad": (_i, [_vp, ctypes.c_long, _i, _i, ctypes.POINTER(_d), _vp, _i]),
    "hlbm_save": (_i, [_vp, ctypes.c_char_p]),
    "hlbm_load": (_i, [_vp, ctypes.c_char_p]),
    "hlbm_server_create": (_i, [ctypes.POINTER(_vp), ctypes.c_size_t, _i, _i, _vp]),
    "hlbm_server_set_refinement": (_i, [_vp, _i, _d]),
    "hlbm_server_set_priority": (_i, [_vp, _d]),
    "hlbm_server_submit": (_i, [_vp, ctypes.POINTER(hlbm_request), ctypes.POINTER(ctypes.c_uint64)]),
    "hlbm_server_pump": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "hlbm_server_poll": (_i, [_vp, ctypes.POINTER(hlbm_result), _i, ctypes.POINTER(_i)]),
    "hlbm_server_cancel": (_i, [_vp, ctypes.c_uint64]),
    "hlbm_server_info": (_i, [_vp, ctypes.POINTER(hlbm_server_stats)]),
    "hlbm_server_inject_alloc_failures": (_i, [_vp, _i]),
    "hlbm_server_destroy": (None, [_vp]),
    "hlbm_reduce_series": (_i, [_vp, ctypes.c_long, _i, _vp, _i]),
    "hlbm_reduce_noalloc": (_i, [_i, _i, _i, _i, _i, ctypes.POINTER(_i), _d, ctypes.POINTER(_d), _d, _i, _vp,
                                 _vp, _vp, ctypes.POINTER(hlbm_stats), _vp]),
    "hlbm_strerror": (ctypes.c_char_p, [_i]),
    "hlbm_last_cuda_error": (ctypes.c_char_p, []),
}


def _lib():
    """Load libhlbm.so (raises if it is missing: there is no fallback)."""
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhlbm.so is not built (%s); run `python -m paper_2310_14746_gb300.build`"
                               % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _L = lib
    return _L


def library():
    """The loaded ctypes library (for symbol checks and direct calls)."""
    return _lib()


def _strerror(status):
    return _lib().hlbm_strerror(int(status)).decode()


def _check(status, call):
    if status != HLBM_OK:
        raise HlbmError(status, call)


def _ptr(buf, dtype):
    """(pointer, on_device) of a torch tensor / numpy array / raw int pointer of dtype."""
    if isinstance(buf, int):
        return buf, 1
    if isinstance(buf, np.ndarray):
        if buf.dtype != dtype or not buf.flags.c_contiguous:
            raise TypeError("expected a C-contiguous %s array" % np.dtype(dtype))
        return buf.ctypes.data, 0
    import torch
    if isinstance(buf, torch.Tensor):
        tdt = {np.float32: torch.float32, np.float64: torch.float64}[np.dtype(dtype).type]
        if buf.dtype != tdt or not buf.is_contiguous():
            raise TypeError("expected a contiguous %s tensor" % tdt)
        return buf.data_ptr(), 1 if buf.is_cuda else 0
    raise TypeError("unsupported buffer type %r" % type(buf))


def current_stream():
    """torch's current CUDA stream as a raw cudaStream_t (int)."""
    import torch
    return torch.cuda.current_stream().cuda_stream


# ---- C-ABI mirrors ----------------------------------------------------------

def hlbm_create(velset, nx, ny, nz, storage=HLBM_F32, pattern=HLBM_TWO_LATTICE, stream=None):
    h = _vp()
    st = current_stream() if stream is None else stream
    _check(_lib().hlbm_create(ctypes.byref(h), velset, nx, ny, nz, storage, pattern, st), "hlbm_create")
    return h.value


def hlbm_destroy(h):
    _lib().hlbm_destroy(h)


def hlbm_release_scratch(h):
    _check(_lib().hlbm_release_scratch(h), "hlbm_release_scratch")


def hlbm_set_stream(h, stream):
    _check(_lib().hlbm_set_stream(h, stream), "hlbm_set_stream")


def hlbm_set_relaxation(h, tau):
    _check(_lib().hlbm_set_relaxation(h, float(tau)), "hlbm_set_relaxation")


def hlbm_set_porosity(h, varpi):
    p, dev = _ptr(varpi, np.float32)
    _check(_lib().hlbm_set_porosity(h, p, dev), "hlbm_set_porosity")


def hlbm_set_porosity_tensor(h, varpi3):
    p, dev = _ptr(varpi3, np.float32)
    _check(_lib().hlbm_set_porosity_tensor(h, p, dev), "hlbm_set_porosity_tensor")


def hlbm_set_solid_mask(h, solid):
    """solid: uint8 numpy array (host) or uint8 CUDA tensor, nonzero = solid; None removes the mask."""
    if solid is None:
        _check(_lib().hlbm_set_solid_mask(h, None, 0), "hlbm_set_solid_mask")
        return
    if isinstance(solid, np.ndarray):
        a = np.ascontiguousarray(solid, dtype=np.uint8)
        _check(_lib().hlbm_set_solid_mask(h, a.ctypes.data, 0), "hlbm_set_solid_mask")
        return
    import torch
    if not (isinstance(solid, torch.Tensor) and solid.dtype == torch.uint8 and solid.is_contiguous()):
        raise TypeError("expected a contiguous uint8 array or CUDA tensor")
    _check(_lib().hlbm_set_solid_mask(h, solid.data_ptr(), 1 if solid.is_cuda else 0), "hlbm_set_solid_mask")


def hlbm_porosity_from_permeability(K, nu, tau):
    K = np.ascontiguousarray(K, dtype=np.float32)
    out = np.empty_like(K)
    _check(_lib().hlbm_porosity_from_permeability(K.ctypes.data, float(nu), float(tau), out.ctypes.data,
                                                  K.size), "hlbm_porosity_from_permeability")
    return out


def hlbm_set_force(h, Fx, Fy, Fz=0.0):
    _check(_lib().hlbm_set_force(h, float(Fx), float(Fy), float(Fz)), "hlbm_set_force")


def hlbm_set_boundary(h, axis, kind):
    _check(_lib().hlbm_set_boundary(h, axis, kind), "hlbm_set_boundary")


def hlbm_set_homogenization(h, form):
    _check(_lib().hlbm_set_homogenization(h, int(form)), "hlbm_set_homogenization")


def hlbm_set_step_kernel(h, variant):
    _check(_lib().hlbm_set_step_kernel(h, int(variant)), "hlbm_set_step_kernel")


def hlbm_set_storage_scale(h, s):
    _check(_lib().hlbm_set_storage_scale(h, float(s)), "hlbm_set_storage_scale")


def hlbm_init_equilibrium(h, rho0=1.0, ux=0.0, uy=0.0, uz=0.0):
    _check(_lib().hlbm_init_equilibrium(h, float(rho0), float(ux), float(uy), float(uz)),
           "hlbm_init_equilibrium")


def hlbm_set_populations(h, f):
    p, dev = _ptr(f, np.float64)
    _check(_lib().hlbm_set_populations(h, p, dev), "hlbm_set_populations")


def hlbm_get_populations(h, out):
    p, dev = _ptr(out, np.float64)
    _check(_lib().hlbm_get_populations(h, p, dev), "hlbm_get_populations")
    return out


def hlbm_step(h, nsteps):
    _check(_lib().hlbm_step(h, int(nsteps)), "hlbm_step")


def hlbm_get_step(h):
    s = ctypes.c_longlong(0)
    _check(_lib().hlbm_get_step(h, ctypes.byref(s)), "hlbm_get_step")
    return s.value


def hlbm_moments(h, rho, u):
    """FP32 rho / u (either may be None) into host arrays or CUDA tensors (both alike)."""
    dev = None
    ptrs = []
    for b in (rho, u):
        if b is None:
            ptrs.append(None)
            continue
        p, d = _ptr(b, np.float32)
        if dev is not None and d != dev:
            raise TypeError("rho and u must both be host or both be device buffers")
        dev = d
        ptrs.append(p)
    _check(_lib().hlbm_moments(h, ptrs[0], ptrs[1], dev or 0), "hlbm_moments")


def hlbm_moments_f64(h, rho, u):
    dev = None
    ptrs = []
    for b in (rho, u):
        if b is None:
            ptrs.append(None)
            continue
        p, d = _ptr(b, np.float64)
        if dev is not None and d != dev:
            raise TypeError("rho and u must both be host or both be device buffers")
        dev = d
        ptrs.append(p)
    _check(_lib().hlbm_moments_f64(h, ptrs[0], ptrs[1], dev or 0), "hlbm_moments_f64")


def hlbm_reduce(h):
    st = hlbm_stats()
    _check(_lib().hlbm_reduce(h, ctypes.byref(st)), "hlbm_reduce")
    return st.as_dict()


def hlbm_reduce_series(h, nsamples, every, out):
    """Writes nsamples records of the 8 FP64 diagnostics into out (float64 numpy array or CUDA
    tensor of 8*nsamples values); record k is the state k*every steps after the call began."""
    p, dev = _ptr(out, np.float64)
    _check(_lib().hlbm_reduce_series(h, int(nsamples), int(every), p, dev), "hlbm_reduce_series")


def hlbm_adjoint_flux_grad(h, nsteps, ckpt_every, plane_x, grad):
    """Returns J; writes dJ/dvarpi into grad (float32 numpy array or CUDA tensor)."""
    p, dev = _ptr(grad, np.float32)
    J = _d(0.0)
    _check(_lib().hlbm_adjoint_flux_grad(h, int(nsteps), int(ckpt_every), int(plane_x), ctypes.byref(J), p, dev),
           "hlbm_adjoint_flux_grad")
    return J.value


def hlbm_save(h, path):
    _check(_lib().hlbm_save(h, os.fsencode(path)), "hlbm_save")


def hlbm_load(h, path):
    _check(_lib().hlbm_load(h, os.fsencode(path)), "hlbm_load")


def hlbm_server_create(mem_budget, storage=HLBM_F16DEV, check_every=100, stream=None):
    h = _vp()
    st = current_stream() if stream is None else stream
    _check(_lib().hlbm_server_create(ctypes.byref(h), int(mem_budget), storage, check_every, st),
           "hlbm_server_create")
    return h.value


def hlbm_server_set_priority(s, backfill):
    _check(_lib().hlbm_server_set_priority(s, float(backfill)), "hlbm_server_set_priority")


def hlbm_server_set_refinement(s, enable, floor_coef):
    _check(_lib().hlbm_server_set_refinement(s, int(bool(enable)), float(floor_coef)), "hlbm_server_set_refinement")


def hlbm_server_submit(s, req):
    rid = ctypes.c_uint64(0)
    _check(_lib().hlbm_server_submit(s, ctypes.byref(req), ctypes.byref(rid)), "hlbm_server_submit")
    return rid.value


def hlbm_server_pump(s):
    a, w = _i(0), _i(0)
    _check(_lib().hlbm_server_pump(s, ctypes.byref(a), ctypes.byref(w)), "hlbm_server_pump")
    return a.value, w.value


def hlbm_server_poll(s, max_results=1024):
    buf = (hlbm_result * max_results)()
    n = _i(0)
    _check(_lib().hlbm_server_poll(s, buf, max_results, ctypes.byref(n)), "hlbm_server_poll")
    return [buf[k].as_dict() for k in range(n.value)]


def hlbm_server_cancel(s, rid):
    _check(_lib().hlbm_server_cancel(s, int(rid)), "hlbm_server_cancel")


def hlbm_server_info(s):
    st = hlbm_server_stats()
    _check(_lib().hlbm_server_info(s, ctypes.byref(st)), "hlbm_server_info")
    return st.as_dict()


def hlbm_server_inject_alloc_failures(s, n):
    _check(_lib().hlbm_server_inject_alloc_failures(s, int(n)), "hlbm_server_inject_alloc_failures")


def hlbm_server_destroy(s):
    _lib().hlbm_server_destroy(s)


def hlbm_reduce_noalloc(velset, nx, ny, nz, storage, bc, tau, F, storage_scale, f, u_prev, stream=None,
                        form=0, varpi=None):
    """Diagnostics without any device allocation; f, u_prev and (for the drag form) varpi are
    device buffers (CUDA tensors or raw pointers) the caller owns. Returns the stats dict."""
    def ptr(t):
        return None if t is None else (t if isinstance(t, int) else t.data_ptr())
    st = hlbm_stats()
    b = (_i * 3)(*bc)
    FF = (_d * 3)(*F)
    s = current_stream() if stream is None else stream
    _check(_lib().hlbm_reduce_noalloc(velset, nx, ny, nz, storage, b, float(tau), FF, float(storage_scale), int(form),
                                      ptr(varpi), ptr(f), ptr(u_prev), ctypes.byref(st), s), "hlbm_reduce_noalloc")
    return st.as_dict()


def hlbm_strerror(status):
    return _strerror(status)


def hlbm_last_cuda_error():
    return _lib().hlbm_last_cuda_error().decode()


# ---- convenience wrapper ------------------------------------------------------

class Lattice:
    """Owning wrapper around an hlbm_t handle (argument marshalling only)."""

    def __init__(self, velset, nx, ny, nz=1, storage=HLBM_F32, pattern=HLBM_TWO_LATTICE, stream=None):
        self.q, self.nx, self.ny, self.nz = velset, nx, ny, nz
        self.storage, self.pattern = storage, pattern
        self.h = hlbm_create(velset, nx, ny, nz, storage, pattern, stream)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def cells(self):
        return self.nx * self.ny * self.nz

    def close(self):
        if self.h:
            hlbm_destroy(self.h)
            self.h = None

    def release_scratch(self):
        """Return the handle's cached scratch memory (hlbm_release_scratch)."""
        hlbm_release_scratch(self.h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_relaxation(self, tau):
        hlbm_set_relaxation(self.h, tau)

    def set_porosity(self, varpi):
        hlbm_set_porosity(self.h, varpi)

    def set_solid_mask(self, solid):
        hlbm_set_solid_mask(self.h, solid)

    def set_porosity_tensor(self, varpi3):
        hlbm_set_porosity_tensor(self.h, varpi3)

    def set_force(self, Fx, Fy=0.0, Fz=0.0):
        hlbm_set_force(self.h, Fx, Fy, Fz)

    def set_boundary(self, axis, kind):
        hlbm_set_boundary(self.h, axis, kind)

    def set_storage_scale(self, s):
        hlbm_set_storage_scale(self.h, s)

    def set_homogenization(self, form):
        hlbm_set_homogenization(self.h, form)

    def set_step_kernel(self, variant):
        hlbm_set_step_kernel(self.h, variant)

    def init_equilibrium(self, rho0=1.0, u0=(0.0, 0.0, 0.0)):
        hlbm_init_equilibrium(self.h, rho0, *u0)

    def set_populations(self, f):
        hlbm_set_populations(self.h, f)

    def get_populations(self):
        out = np.empty((self.q,) + self.shape, dtype=np.float64)
        return hlbm_get_populations(self.h, out)

    def step(self, n=1):
        hlbm_step(self.h, n)

    @property
    def steps_taken(self):
        return hlbm_get_step(self.h)

    def moments(self, f64=False):
        """Host (rho, u) arrays; FP64 outputs when f64."""
        dt = np.float64 if f64 else np.float32
        rho = np.empty(self.shape, dtype=dt)
        u = np.empty((3,) + self.shape, dtype=dt)
        (hlbm_moments_f64 if f64 else hlbm_moments)(self.h, rho, u)
        return rho, u

    def reduce(self):
        return hlbm_reduce(self.h)

    def reduce_series(self, nsamples, every=1, out=None):
        """(nsamples, 8) FP64 diagnostics records, one every `every` steps from the current state
        (columns in the order of STAT_KEYS); out may be a CUDA tensor (asynchronous)."""
        if out is None:
            out = np.empty((nsamples, 8), dtype=np.float64)
        hlbm_reduce_series(self.h, nsamples, every, out)
        return out

    def adjoint_flux_grad(self, nsteps, ckpt_every=45, plane_x=None, grad=None):
        """(J, dJ/dvarpi) of the outflow flux through x = plane_x (default nx-1) after nsteps."""
        if grad is None:
            grad = np.empty(self.shape, dtype=np.float32)
        px = self.nx - 1 if plane_x is None else plane_x
        J = hlbm_adjoint_flux_grad(self.h, nsteps, ckpt_every, px, grad)
        return J, grad

    def save(self, path):
        hlbm_save(self.h, path)

    def load(self, path):
        hlbm_load(self.h, path)
