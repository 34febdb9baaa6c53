"""Plain FP64 CPU oracle of the filtered LES-LB-MHD time step (arXiv:1705.09807).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The product path
(the CUDA library and its binding) never imports or links it.  Its one import from the
product's package is the seeded input generator ``paper_1705_09807_gb300.inputs`` (used by
``closure.init_params`` for its random weights), which holds none of the method's arithmetic.

The arithmetic lives in ``lbmhd_oracle.c`` (plain C, binary64, ``-O2 -ffp-contract=off``);
this module builds it with gcc on first use and marshals numpy arrays through ctypes.
Array layouts: fields ``[ny, nx]`` (x fastest); ``f[9, ny, nx]``; ``g[2, 9, ny, nx]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbmhd_oracle.c")
_LIB = os.path.join(_HERE, "liblbmhd_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (idempotent unless ``force``); returns the .so path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_tables.argtypes = [_I, _I, _D, _D, _D, _D, _D]
            lib.oracle_feq.argtypes = [ctypes.c_double] * 5 + [_D]
            lib.oracle_geq.argtypes = [ctypes.c_double] * 4 + [_D]
            lib.oracle_meq.argtypes = [ctypes.c_double, _D, _D, _D, _D, ctypes.c_double, _D]
            lib.oracle_neq.argtypes = [ctypes.c_double, _D, _D, _D, _D, ctypes.c_double, _D]
            lib.oracle_step.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, _D, _D, ctypes.c_int,
                                        ctypes.c_int]
            lib.oracle_step_corrected.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_int, _D, _D,
                                                  ctypes.c_int, ctypes.c_int, _D]
            lib.oracle_collide_cell.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int, _D, _D,
                                                ctypes.c_int, ctypes.c_int, _D, _D]
            lib.oracle_init.argtypes = [ctypes.c_int, ctypes.c_int] + [_D] * 7
            lib.oracle_moments.argtypes = [ctypes.c_int, ctypes.c_int] + [_D] * 7
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _arr(x, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def tables() -> dict:
    """The lattice vectors, weights, T, T_m and the inverses the oracle computes."""
    lib = _load()
    cx = (ctypes.c_int * 9)()
    cy = (ctypes.c_int * 9)()
    w = np.zeros(9)
    T, Tm, Ti, Tmi = (np.zeros((9, 9)) for _ in range(4))
    _check(lib.oracle_tables(cx, cy, _p(w), _p(T), _p(Tm), _p(Ti), _p(Tmi)), "tables")
    return {"cx": np.array(list(cx)), "cy": np.array(list(cy)), "w": w, "T": T, "Tm": Tm,
            "Tinv": Ti, "Tminv": Tmi}


def feq(rho, ux, uy, bx, by) -> np.ndarray:
    """Eq. feq at one point."""
    out = np.zeros(9)
    _load().oracle_feq(rho, ux, uy, bx, by, _p(out))
    return out


def geq(ux, uy, bx, by) -> np.ndarray:
    """Eq. geq at one point, shape [2, 9]."""
    out = np.zeros(18)
    _load().oracle_geq(ux, uy, bx, by, _p(out))
    return out.reshape(2, 9)


def meq(rho, J, B, gJ, gB, delta) -> np.ndarray:
    """Filtered fluid equilibrium moments; gJ[a][beta] = d_beta J_a."""
    J, B, gJ, gB = _arr(J, 2), _arr(B, 2), _arr(gJ, 4), _arr(gB, 4)
    out = np.zeros(9)
    _load().oracle_meq(rho, _p(J), _p(B), _p(gJ), _p(gB), delta * delta / 12.0, _p(out))
    return out


def neq(rho, J, B, gJ, gB, delta) -> np.ndarray:
    """Filtered magnetic equilibrium moments, shape [2, 9]."""
    J, B, gJ, gB = _arr(J, 2), _arr(B, 2), _arr(gJ, 4), _arr(gB, 4)
    out = np.zeros(18)
    _load().oracle_neq(rho, _p(J), _p(B), _p(gJ), _p(gB), delta * delta / 12.0, _p(out))
    return out.reshape(2, 9)


def init(rho, ux, uy, bx, by):
    """Equilibrium populations (f [9,ny,nx], g [2,9,ny,nx]) for the given fields."""
    rho, ux, uy, bx, by = (_arr(a) for a in (rho, ux, uy, bx, by))
    ny, nx = rho.shape
    f = np.zeros((9, ny, nx))
    g = np.zeros((2, 9, ny, nx))
    _check(_load().oracle_init(nx, ny, _p(rho), _p(ux), _p(uy), _p(bx), _p(by), _p(f), _p(g)),
           "init")
    return f, g


def step(f, g, s, s_m, delta, nsteps, stencil=0, nthreads=1):
    """Return (f, g) advanced by ``nsteps`` steps (inputs are not modified)."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    g = np.array(g, dtype=np.float64, order="C", copy=True)
    ny, nx = f.shape[1:]
    s = _arr(s, 9)
    _check(_load().oracle_step(nx, ny, _p(s), s_m, delta, stencil, _p(f), _p(g), nsteps,
                               nthreads), "step")
    return f, g


def step_inplace(f, g, s, s_m, delta, nsteps, stencil=0, nthreads=1) -> None:
    """``step`` advancing ``f`` and ``g`` in place (C-contiguous float64 arrays, no copy): for
    timing the oracle on large grids, where a copy of the state would cost as much as a step."""
    if not (f.dtype == np.float64 and g.dtype == np.float64 and f.flags["C_CONTIGUOUS"]
            and g.flags["C_CONTIGUOUS"] and f.flags["WRITEABLE"] and g.flags["WRITEABLE"]):
        raise ValueError("step_inplace needs writeable C-contiguous float64 arrays")
    ny, nx = f.shape[1:]
    s = _arr(s, 9)
    _check(_load().oracle_step(nx, ny, _p(s), s_m, delta, stencil, _p(f), _p(g), nsteps,
                               nthreads), "step")


def step_corrected(f, g, s, s_m, delta, nsteps, corr, stencil=0, nthreads=1):
    """``step`` with a fixed additive correction corr[4, ny, nx] of the four subgrid terms
    (xy stress, normal-stress difference, trace, electric field) at every cell and step."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    g = np.array(g, dtype=np.float64, order="C", copy=True)
    ny, nx = f.shape[1:]
    s = _arr(s, 9)
    corr = _arr(corr, (4, ny, nx))
    _check(_load().oracle_step_corrected(nx, ny, _p(s), s_m, delta, stencil, _p(f), _p(g), nsteps,
                                         nthreads, _p(corr)), "step_corrected")
    return f, g


def collide_cell(f, g, s, s_m, delta, x, y, stencil=0):
    """Post-collision (f* [9], g* [2,9]) of cell (x, y) of the current state."""
    f = _arr(f)
    g = _arr(g)
    ny, nx = f.shape[1:]
    s = _arr(s, 9)
    fs = np.zeros(9)
    gs = np.zeros(18)
    _check(_load().oracle_collide_cell(nx, ny, _p(s), s_m, delta, stencil, _p(f), _p(g), x, y,
                                       _p(fs), _p(gs)), "collide_cell")
    return fs, gs.reshape(2, 9)


def moments(f, g):
    """(rho, ux, uy, bx, by) of the current populations, each [ny, nx]."""
    f = _arr(f)
    g = _arr(g)
    ny, nx = f.shape[1:]
    outs = [np.zeros((ny, nx)) for _ in range(5)]
    _check(_load().oracle_moments(nx, ny, _p(f), _p(g), *(_p(o) for o in outs)), "moments")
    return tuple(outs)


def srt_rates(nu: float) -> np.ndarray:
    """All nine fluid rates equal to s = 1/(3 nu + 1/2) (Sec. 3 SRT; nu relation of Sec. 2)."""
    return np.full(9, 1.0 / (3.0 * nu + 0.5))


def rate_from_diffusivity(d: float) -> float:
    """s = 1/(3 d + 1/2), the inverse of nu = 1/(3 s) - 1/6 (Sec. 2)."""
    return 1.0 / (3.0 * d + 0.5)
