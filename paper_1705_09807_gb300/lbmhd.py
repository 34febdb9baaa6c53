"""Python binding of liblbmhd.so (the C ABI in include/lbmhd.h): argument marshalling only.

Every step of the time-stepping path runs in the library's CUDA kernels; this module never
computes any part of it.  If the shared library is missing it raises instead of falling back
to anything else.  Host arrays are numpy float64 ``[ny, nx]``; device arrays are torch CUDA
float64 tensors (PyTorch only supplies device memory and the stream).
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbmhd.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "lbmhd.h")

LBMHD_OK = 0
LBMHD_ERR_INVALID = -1
LBMHD_ERR_CUDA = -2
LBMHD_ERR_OOM = -3
LBMHD_ERR_UNSTABLE = -4
LBMHD_FP64 = 0
LBMHD_FP32 = 1
LBMHD_FP16 = 2
LBMHD_FP16_REL = 3
LBMHD_ERR_TIMEOUT = -5
LBMHD_GRAD_CENTRAL = 0
LBMHD_GRAD_ISOTROPIC = 1
LBMHD_NDIAG = 10

DIAG_NAMES = ("mass", "jx", "jy", "bx", "by", "e_kin", "e_mag", "max_div_b_iso",
              "max_div_b_central", "max_grad_b_iso")


class LbmhdParams(ctypes.Structure):
    """Mirror of ``lbmhd_params`` (include/lbmhd.h)."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("s", ctypes.c_double * 9),
                ("s_m", ctypes.c_double), ("delta", ctypes.c_double),
                ("precision", ctypes.c_int), ("grad_stencil", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p)]


class LbmhdError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"lbmhd error {code}: {message}")
        self.code = code


class LbmhdUnstable(LbmhdError):
    def __init__(self, code, message, values):
        super().__init__(code, message)
        self.values = values


_lib = None
_lock = threading.Lock()
_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_H = ctypes.c_void_p


def load_library(path: str | None = None):
    """Load liblbmhd.so (once).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with `python -m paper_1705_09807_gb300.build` "
                               "(there is no fallback implementation)")
        lib = ctypes.CDLL(p)
        P = ctypes.POINTER(LbmhdParams)
        sig = {
            "lbmhd_params_srt": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_int]),
            "lbmhd_init": (ctypes.c_int, [ctypes.POINTER(_H), P, _D, _D, _D, _D, _D]),
            "lbmhd_init_device": (ctypes.c_int, [ctypes.POINTER(_H), P] + [ctypes.c_void_p] * 5),
            "lbmhd_step": (ctypes.c_int, [_H, ctypes.c_int]),
            "lbmhd_moments": (ctypes.c_int, [_H, _D, _D, _D, _D, _D]),
            "lbmhd_moments_device": (ctypes.c_int, [_H] + [ctypes.c_void_p] * 5),
            "lbmhd_get_populations": (ctypes.c_int, [_H, _D]),
            "lbmhd_diagnostics": (ctypes.c_int, [_H, _D]),
            "lbmhd_state_bytes": (ctypes.c_size_t, [_H]),
            "lbmhd_get_state": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_size_t]),
            "lbmhd_set_state": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_size_t]),
            "lbmhd_get_stream": (ctypes.c_void_p, [_H]),
            "lbmhd_diagnostics_fields_noalloc": (ctypes.c_int, [ctypes.c_void_p] * 5 + [
                ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
            "lbmhd_block_mean_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
            "lbmhd_energy_spectrum_work_bytes": (ctypes.c_size_t, [ctypes.c_int]),
            "lbmhd_energy_spectrum_device": (ctypes.c_int, [ctypes.c_void_p] * 4 + [
                ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_size_t, ctypes.c_void_p]),
            "lbmhd_energy_spectrum": (ctypes.c_int, [_H, ctypes.c_int, _D, _D]),
            "lbmhd_launch_count": (ctypes.c_uint64, [_H]),
            "lbmhd_probe_fp64_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _D]),
            "lbmhd_ensemble_create": (ctypes.c_int, [ctypes.POINTER(_H), ctypes.c_int, P,
                                                     ctypes.POINTER(_D), ctypes.c_void_p]),
            "lbmhd_ensemble_step": (ctypes.c_int, [_H, ctypes.c_int]),
            "lbmhd_ensemble_set_schedule": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int]),
            "lbmhd_ensemble_get_schedule": (ctypes.c_int, [_H] + [ctypes.POINTER(ctypes.c_int)] * 4),
            "lbmhd_ensemble_autotune": (ctypes.c_int, [_H, ctypes.c_int, _D]),
            "lbmhd_ensemble_sync": (ctypes.c_int, [_H]),
            "lbmhd_ensemble_member": (ctypes.c_void_p, [_H, ctypes.c_int]),
            "lbmhd_ensemble_size": (ctypes.c_int, [_H]),
            "lbmhd_ensemble_get_stream": (ctypes.c_void_p, [_H]),
            "lbmhd_ensemble_launch_count": (ctypes.c_uint64, [_H]),
            "lbmhd_ensemble_last_error": (ctypes.c_char_p, [_H]),
            "lbmhd_ensemble_free": (None, [_H]),
            "lbmhd_set_correction_device": (ctypes.c_int, [_H, ctypes.c_void_p]),
            "lbmhd_test_skip_row_copy": (ctypes.c_int, [_H, ctypes.c_int]),
            "lbmhd_set_closure": (ctypes.c_int, [_H, ctypes.c_void_p]),
            "lbmhd_closure_correction_device": (ctypes.c_int, [_H, ctypes.c_void_p]),
            "lbmhd_closure_num_params": (ctypes.c_int, []),
            "lbmhd_closure_create": (ctypes.c_int, [ctypes.POINTER(_H), _F, _F, _F]),
            "lbmhd_closure_get_params": (ctypes.c_int, [_H, _F]),
            "lbmhd_closure_set_params": (ctypes.c_int, [_H, _F]),
            "lbmhd_closure_training_pair": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                           ctypes.c_double, ctypes.c_void_p,
                                                           ctypes.c_void_p, ctypes.c_void_p]),
            "lbmhd_closure_features": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                                      ctypes.c_void_p, ctypes.c_void_p]),
            "lbmhd_closure_gradient": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                      ctypes.c_int, ctypes.c_int, _F, _D]),
            "lbmhd_closure_train_step": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                        ctypes.c_int, ctypes.c_int, ctypes.c_float, _D]),
            "lbmhd_closure_forward": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
            "lbmhd_closure_last_error": (ctypes.c_char_p, [_H]),
            "lbmhd_closure_test_skip_mma": (ctypes.c_int, [_H, ctypes.c_int]),
            "lbmhd_closure_free": (None, [_H]),
            "lbmhd_step_count": (ctypes.c_int64, [_H]),
            "lbmhd_last_error": (ctypes.c_char_p, [_H]),
            "lbmhd_free": (None, [_H]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def header_functions(path: str = HEADER_PATH) -> list:
    """Names of the functions the public header declares."""
    with open(path) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbmhd_[a-z_0-9]+)\s*\(", text)))


def _err(h) -> str:
    m = load_library().lbmhd_last_error(h)
    return m.decode() if m else ""


def _check(rc: int, h=None) -> None:
    if rc != LBMHD_OK:
        raise LbmhdError(rc, _err(h))


def _host(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected an array of shape {shape}, got {a.shape}")
    return a


def _dptr(t, n: int) -> int:
    """Data pointer of a contiguous CUDA float64 tensor with n elements."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous() and t.numel() == n):
        raise ValueError("expected a contiguous CUDA float64 tensor of matching size")
    return t.data_ptr()


# ---------------------------------------------------------------- functions of the C ABI
def lbmhd_params_srt(nx, ny, nu, eta, delta, precision=LBMHD_FP64) -> LbmhdParams:
    p = LbmhdParams()
    _check(load_library().lbmhd_params_srt(ctypes.byref(p), nx, ny, nu, eta, delta, precision))
    return p


def make_params(nx, ny, s, s_m, delta, precision=LBMHD_FP64, grad_stencil=LBMHD_GRAD_CENTRAL,
                cuda_stream=None) -> LbmhdParams:
    p = LbmhdParams()
    p.nx, p.ny = nx, ny
    s = np.asarray(s, dtype=np.float64).reshape(9)
    for j in range(9):
        p.s[j] = float(s[j])
    p.s_m, p.delta = float(s_m), float(delta)
    p.precision, p.grad_stencil = int(precision), int(grad_stencil)
    p.cuda_stream = cuda_stream
    return p


def lbmhd_init(p: LbmhdParams, rho, ux, uy, bx, by):
    shape = (p.ny, p.nx)
    arrs = [_host(a, shape) for a in (rho, ux, uy, bx, by)]
    h = _H()
    rc = load_library().lbmhd_init(ctypes.byref(h), ctypes.byref(p),
                                   *(a.ctypes.data_as(_D) for a in arrs))
    _check(rc, None)
    return h


def lbmhd_init_device(p: LbmhdParams, rho, ux, uy, bx, by):
    n = p.nx * p.ny
    h = _H()
    rc = load_library().lbmhd_init_device(ctypes.byref(h), ctypes.byref(p),
                                          *(_dptr(t, n) for t in (rho, ux, uy, bx, by)))
    _check(rc, None)
    return h


def lbmhd_step(h, nsteps: int) -> None:
    _check(load_library().lbmhd_step(h, int(nsteps)), h)


def lbmhd_moments(h, ny: int, nx: int, out=None):
    """(rho, ux, uy, bx, by) as host arrays: new pageable arrays, or the five C-contiguous
    float64 [ny, nx] arrays of `out` (page-locked ones are written by the kernel directly)."""
    if out is None:
        outs = [np.empty((ny, nx)) for _ in range(5)]
    else:
        outs = list(out)
        if len(outs) != 5 or not all(isinstance(o, np.ndarray) and o.dtype == np.float64 and
                                     o.shape == (ny, nx) and o.flags.c_contiguous for o in outs):
            raise ValueError(f"out must be five C-contiguous float64 arrays of shape {(ny, nx)}")
    _check(load_library().lbmhd_moments(h, *(o.ctypes.data_as(_D) for o in outs)), h)
    return tuple(outs)


def lbmhd_moments_device(h, outs) -> None:
    n = outs[0].numel()
    _check(load_library().lbmhd_moments_device(h, *(_dptr(t, n) for t in outs)), h)


def lbmhd_get_populations(h, ny: int, nx: int) -> np.ndarray:
    out = np.empty((27, ny, nx))
    _check(load_library().lbmhd_get_populations(h, out.ctypes.data_as(_D)), h)
    return out


def lbmhd_diagnostics(h) -> np.ndarray:
    out = np.zeros(LBMHD_NDIAG)
    rc = load_library().lbmhd_diagnostics(h, out.ctypes.data_as(_D))
    if rc == LBMHD_ERR_UNSTABLE:
        raise LbmhdUnstable(rc, _err(h), out)
    _check(rc, h)
    return out


def lbmhd_diagnostics_fields_noalloc(fields, out, stream=None) -> None:
    """Diagnostics of five device moment fields [ny, nx] into the device tensor ``out``
    (LBMHD_NDIAG + 1 float64: the values, then the instability flag), allocating nothing on
    the device; for callers that cannot allocate (see include/lbmhd.h)."""
    ny, nx = fields[0].shape
    ptrs = [_dptr(t, nx * ny) for t in fields]
    rc = load_library().lbmhd_diagnostics_fields_noalloc(*ptrs, nx, ny,
                                                         _dptr(out, LBMHD_NDIAG + 1), stream)
    _check(rc, None)


def lbmhd_block_mean_device(field, r: int, out, stream=None) -> None:
    """r x r block means of a CUDA float64 [ny, nx] tensor into ``out`` [ny/r, nx/r]."""
    ny, nx = field.shape
    if nx % r or ny % r:
        raise ValueError("r must divide both grid sides")
    _check(load_library().lbmhd_block_mean_device(_dptr(field, nx * ny), nx, ny, r,
                                                  _dptr(out, (nx // r) * (ny // r)), stream))


def lbmhd_energy_spectrum_device(ux, uy, bx, by, nbins: int, e_kin, e_mag, work, stream=None):
    """Shell spectra of square CUDA float64 fields into CUDA float64 e_kin, e_mag [nbins];
    ``work`` is a CUDA byte tensor of at least lbmhd_energy_spectrum_work_bytes(n) bytes."""
    n = ux.shape[0]
    lib = load_library()
    ptrs = [_dptr(t, n * n) for t in (ux, uy, bx, by)]
    _check(lib.lbmhd_energy_spectrum_device(*ptrs, n, nbins, _dptr(e_kin, nbins), _dptr(e_mag, nbins),
                                            work.data_ptr(), work.numel() * work.element_size(),
                                            stream))


def lbmhd_energy_spectrum_work_bytes(n: int) -> int:
    return int(load_library().lbmhd_energy_spectrum_work_bytes(n))


def lbmhd_energy_spectrum(h, nbins: int):
    ek = np.zeros(nbins)
    em = np.zeros(nbins)
    _check(load_library().lbmhd_energy_spectrum(h, nbins, ek.ctypes.data_as(_D), em.ctypes.data_as(_D)), h)
    return ek, em


def lbmhd_state_bytes(h) -> int:
    return int(load_library().lbmhd_state_bytes(h))


def lbmhd_get_state(h) -> np.ndarray:
    buf = np.empty(lbmhd_state_bytes(h), dtype=np.uint8)
    _check(load_library().lbmhd_get_state(h, buf.ctypes.data, buf.nbytes), h)
    return buf


def lbmhd_set_state(h, buf) -> None:
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(load_library().lbmhd_set_state(h, buf.ctypes.data, buf.nbytes), h)


def lbmhd_test_skip_row_copy(h, enable: bool) -> None:
    _check(load_library().lbmhd_test_skip_row_copy(h, 1 if enable else 0), h)


def lbmhd_get_stream(h) -> int:
    return int(load_library().lbmhd_get_stream(h) or 0)


def lbmhd_launch_count(h) -> int:
    return int(load_library().lbmhd_launch_count(h))


def lbmhd_step_count(h) -> int:
    return int(load_library().lbmhd_step_count(h))


def lbmhd_probe_fp64_fma_rate(iters: int = 4096, repeats: int = 5) -> float:
    """Measured binary64 FMA instructions per second of the current GPU."""
    v = ctypes.c_double(0.0)
    _check(load_library().lbmhd_probe_fp64_fma_rate(iters, repeats, ctypes.byref(v)))
    return v.value


def lbmhd_last_error(h=None) -> str:
    return _err(h)


def lbmhd_free(h) -> None:
    if h is not None and h.value:
        load_library().lbmhd_free(h)


# ---------------------------------------------------------------- convenience wrapper
class Lbmhd:
    """Owns one handle; thin sugar over the functions above."""

    def __init__(self, params: LbmhdParams, rho, ux, uy, bx, by, device: bool = False):
        self.params = params
        self.nx, self.ny = params.nx, params.ny
        self.h = (lbmhd_init_device if device else lbmhd_init)(params, rho, ux, uy, bx, by)

    def step(self, n: int) -> "Lbmhd":
        lbmhd_step(self.h, n)
        return self

    def moments(self, out=None):
        return lbmhd_moments(self.h, self.ny, self.nx, out)

    def moments_device(self, outs):
        lbmhd_moments_device(self.h, outs)

    def populations(self) -> np.ndarray:
        return lbmhd_get_populations(self.h, self.ny, self.nx)

    def diagnostics(self) -> np.ndarray:
        return lbmhd_diagnostics(self.h)

    def spectrum(self, nbins: int):
        return lbmhd_energy_spectrum(self.h, nbins)

    def get_state(self) -> np.ndarray:
        return lbmhd_get_state(self.h)

    def set_state(self, buf) -> None:
        lbmhd_set_state(self.h, buf)

    @property
    def stream(self) -> int:
        return lbmhd_get_stream(self.h)

    @property
    def launches(self) -> int:
        return lbmhd_launch_count(self.h)

    @property
    def steps(self) -> int:
        return lbmhd_step_count(self.h)

    def free(self) -> None:
        if self.h is not None:
            lbmhd_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------- ensembles
class Ensemble:
    """Many independent runs advanced by one launch per step (lbmhd_ensemble_* in the C ABI).
    ``members`` is a list of (params, (rho, ux, uy, bx, by)) with host numpy fields."""

    def __init__(self, members, cuda_stream=None):
        lib = load_library()
        n = len(members)
        self._params = (LbmhdParams * n)(*[p for p, _ in members])
        self._fields = []
        ptrs = (_D * (5 * n))()
        for i, (p, f) in enumerate(members):
            for k, a in enumerate(f):
                a = _host(a, (p.ny, p.nx))
                self._fields.append(a)
                ptrs[5 * i + k] = a.ctypes.data_as(_D)
        self.h = _H()
        rc = lib.lbmhd_ensemble_create(ctypes.byref(self.h), n, self._params, ptrs, cuda_stream)
        if rc != LBMHD_OK:
            raise LbmhdError(rc, (lib.lbmhd_ensemble_last_error(None) or b"").decode())
        self._fields = None
        self.n = n
        self.shapes = [(p.ny, p.nx) for p, _ in members]

    def _check(self, rc):
        if rc != LBMHD_OK:
            raise LbmhdError(rc, (load_library().lbmhd_ensemble_last_error(self.h) or b"").decode())

    def step(self, nsteps: int):
        self._check(load_library().lbmhd_ensemble_step(self.h, int(nsteps)))
        return self

    def set_schedule(self, rows_per_tile: int, persistent: bool):
        self._check(load_library().lbmhd_ensemble_set_schedule(self.h, rows_per_tile, int(persistent)))

    def schedule(self):
        v = [ctypes.c_int() for _ in range(4)]
        self._check(load_library().lbmhd_ensemble_get_schedule(self.h, *(ctypes.byref(x) for x in v)))
        return {"rows_per_tile": v[0].value, "persistent": bool(v[1].value), "tiles": v[2].value,
                "blocks": v[3].value}

    def autotune(self, trial_steps: int = 20) -> float:
        best = ctypes.c_double()
        self._check(load_library().lbmhd_ensemble_autotune(self.h, trial_steps, ctypes.byref(best)))
        return best.value

    def sync(self):
        self._check(load_library().lbmhd_ensemble_sync(self.h))

    def member(self, i: int):
        return _H(load_library().lbmhd_ensemble_member(self.h, i))

    def moments(self, i: int):
        ny, nx = self.shapes[i]
        return lbmhd_moments(self.member(i), ny, nx)

    def populations(self, i: int):
        ny, nx = self.shapes[i]
        return lbmhd_get_populations(self.member(i), ny, nx)

    @property
    def stream(self) -> int:
        return int(load_library().lbmhd_ensemble_get_stream(self.h) or 0)

    @property
    def launches(self) -> int:
        return int(load_library().lbmhd_ensemble_launch_count(self.h))

    def free(self):
        if self.h is not None and self.h.value:
            load_library().lbmhd_ensemble_free(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------- subgrid correction, closure
def lbmhd_set_correction_device(h, corr) -> None:
    """Static correction planes: CUDA float32 tensor [4, ny, nx] (kept alive by the caller), or
    None to detach."""
    ptr = None
    if corr is not None:
        import torch
        if not (corr.is_cuda and corr.dtype == torch.float32 and corr.is_contiguous()):
            raise ValueError("expected a contiguous CUDA float32 tensor [4, ny, nx]")
        ptr = corr.data_ptr()
    _check(load_library().lbmhd_set_correction_device(h, ptr), h)


def _f32(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values")
    return a


class Closure:
    """The learned subgrid correction network (lbmhd_closure_* in the C ABI)."""

    def __init__(self, params, in_scale, out_scale):
        lib = load_library()
        self.n_params = int(lib.lbmhd_closure_num_params())
        p = _f32(params, self.n_params)
        i = _f32(in_scale, 12)
        o = _f32(out_scale, 4)
        self.h = _H()
        rc = lib.lbmhd_closure_create(ctypes.byref(self.h), p.ctypes.data_as(_F), i.ctypes.data_as(_F),
                                      o.ctypes.data_as(_F))
        if rc != LBMHD_OK:
            raise LbmhdError(rc, (lib.lbmhd_closure_last_error(None) or b"").decode())
        self.in_scale, self.out_scale = i, o

    def _check(self, rc):
        if rc != LBMHD_OK:
            raise LbmhdError(rc, (load_library().lbmhd_closure_last_error(self.h) or b"").decode())

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        self._check(load_library().lbmhd_closure_get_params(self.h, out.ctypes.data_as(_F)))
        return out

    def set_params(self, params) -> None:
        p = _f32(params, self.n_params)
        self._check(load_library().lbmhd_closure_set_params(self.h, p.ctypes.data_as(_F)))

    def training_pair(self, fine, r, delta, x, t, work) -> None:
        """fine: CUDA float64 [5, n, n] (rho, ux, uy, bx, by); x [12, m, m], t [4, m, m] float32;
        work: CUDA float64 with at least 9 m^2 elements."""
        n = fine.shape[-1]
        m = n // r
        self._check(load_library().lbmhd_closure_training_pair(
            self.h, _dptr(fine, 5 * n * n), n, r, delta, _dptr32(x, 12 * m * m), _dptr32(t, 4 * m * m),
            _dptr(work, work.numel()) if work.numel() >= 9 * m * m else None))

    def features(self, state, delta, x, analytic=None) -> None:
        m = state.shape[-1]
        self._check(load_library().lbmhd_closure_features(
            self.h, _dptr(state, 5 * m * m), m, delta, _dptr32(x, 12 * m * m),
            None if analytic is None else _dptr32(analytic, 4 * m * m)))

    def gradient(self, x, t):
        b, _, hh, ww = x.shape
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(load_library().lbmhd_closure_gradient(
            self.h, _dptr32(x, x.numel()), _dptr32(t, t.numel()), b, hh, ww, g.ctypes.data_as(_F),
            ctypes.byref(loss)))
        return loss.value, g

    def train_step(self, x, t, lr: float) -> float:
        b, _, hh, ww = x.shape
        loss = ctypes.c_double()
        self._check(load_library().lbmhd_closure_train_step(
            self.h, _dptr32(x, x.numel()), _dptr32(t, t.numel()), b, hh, ww, float(lr), ctypes.byref(loss)))
        return loss.value

    def forward(self, x, out, tensor_cores: bool = True) -> None:
        b, _, hh, ww = x.shape
        self._check(load_library().lbmhd_closure_forward(
            self.h, _dptr32(x, x.numel()), b, hh, ww, _dptr32(out, out.numel()), int(tensor_cores)))

    def test_skip_mma(self, enable: bool) -> None:
        self._check(load_library().lbmhd_closure_test_skip_mma(self.h, 1 if enable else 0))

    def attach(self, h) -> None:
        _check(load_library().lbmhd_set_closure(h, self.h), h)

    def free(self):
        if self.h is not None and self.h.value:
            load_library().lbmhd_closure_free(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def lbmhd_closure_correction_device(h, corr) -> None:
    """The attached closure's correction planes of the current state into corr, a torch CUDA
    float32 tensor [4, ny, nx] (contiguous)."""
    _check(load_library().lbmhd_closure_correction_device(h, _dptr32(corr, corr.numel())), h)


def lbmhd_detach_closure(h) -> None:
    _check(load_library().lbmhd_set_closure(h, None), h)


def _dptr32(t, n: int) -> int:
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous() and t.numel() == n):
        raise ValueError("expected a contiguous CUDA float32 tensor of matching size")
    return t.data_ptr()
