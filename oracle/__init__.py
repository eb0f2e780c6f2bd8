"""Python access to the plain FP64 CPU oracle (``oracle/sph_oracle.c``).

Test infrastructure: only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package.  The CUDA library and its
binding never do.  Arrays are numpy, in the caller's particle order; positions
and velocities are ``(n, dim)`` float64, phase and wall flags ``uint8``.

The equations are those of Sec. II of Wei et al. (two-phase SPH); each C
function documents the equation it restates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


class OrParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int32),
        ("visc_form", C.c_int32),
        ("renorm_every", C.c_int32),
        ("periodic", C.c_int32),
        ("renorm_walls", C.c_int32),
        ("h", C.c_double),
        ("c0", C.c_double),
        ("gamma", C.c_double),
        ("delta", C.c_double),
        ("alpha_s", C.c_double),
        ("cell_size", C.c_double),
        ("g", C.c_double * 3),
        ("rho0", C.c_double * 2),
        ("mu", C.c_double * 2),
        ("mass", C.c_double * 2),
        ("box_lo", C.c_double * 3),
        ("box_hi", C.c_double * 3),
    ]


class OrPiston(C.Structure):
    _fields_ = [
        ("axis", C.c_int32),
        ("ncomp", C.c_int32),
        ("t_end", C.c_double),
        ("amp", C.c_double * 8),
        ("omega", C.c_double * 8),
        ("phase", C.c_double * 8),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over particles) into liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.POINTER
        dp, ip, u8p = P(C.c_double), P(C.c_int32), P(C.c_uint8)
        i64p = P(C.c_int64)
        L.or_W.restype = C.c_double
        L.or_W.argtypes = [C.c_int, C.c_double, C.c_double]
        L.or_dWdr.restype = C.c_double
        L.or_dWdr.argtypes = [C.c_int, C.c_double, C.c_double]
        L.or_eos.restype = C.c_double
        L.or_eos.argtypes = [P(OrParams), C.c_int, C.c_double]
        L.or_eos_inverse.restype = C.c_double
        L.or_eos_inverse.argtypes = [P(OrParams), C.c_int, C.c_double]
        L.or_grid_dims.argtypes = [P(OrParams), ip]
        L.or_cell_ids.restype = C.c_int64
        L.or_cell_ids.argtypes = [P(OrParams), C.c_int64, dp, ip]
        L.or_sort_perm.argtypes = [C.c_int64, ip, i64p]
        for f in (L.or_neighbours_brute, L.or_neighbours_cells):
            f.restype = C.c_int64
            f.argtypes = [P(OrParams), C.c_int64, dp, i64p, ip, C.c_int64]
        L.or_eval.restype = C.c_int
        L.or_eval.argtypes = [P(OrParams), C.c_int64, dp, dp, dp, u8p, u8p, C.c_int,
                              dp, dp, dp, dp, dp, dp]
        L.or_step.restype = C.c_int
        L.or_step.argtypes = [P(OrParams), C.c_int64, dp, dp, dp, u8p, u8p, C.c_double, C.c_int64,
                              P(OrPiston), C.c_double]
        L.or_run.restype = C.c_int
        L.or_run.argtypes = [P(OrParams), C.c_int64, dp, dp, dp, u8p, u8p, C.c_double,
                             C.c_int64, C.c_int64, P(OrPiston), C.c_double]
        for f in (L.or_piston_disp, L.or_piston_vel):
            f.restype = C.c_double
            f.argtypes = [P(OrPiston), C.c_double]
        L.or_diag.argtypes = [P(OrParams), C.c_int64, dp, dp, u8p, u8p, dp]
        L.or_num_threads.restype = C.c_int
        L.or_set_num_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def make_params(p: dict) -> OrParams:
    """Fill the oracle's own parameter struct from a plain dict of values."""
    o = OrParams()
    o.dim = int(p["dim"])
    o.visc_form = int(p.get("visc_form", 0))
    o.renorm_every = int(p.get("renorm_every", 1))
    o.periodic = int(p.get("periodic", 0))
    o.renorm_walls = int(p.get("renorm_walls", 1))
    o.h = p["h"]
    o.c0 = p["c0"]
    o.gamma = p.get("gamma", 7.0)
    o.delta = p["delta"]
    o.alpha_s = p["alpha_s"]
    o.cell_size = p["cell_size"]
    for k in range(3):
        o.g[k] = p["g"][k]
        o.box_lo[k] = p["box_lo"][k]
        o.box_hi[k] = p["box_hi"][k]
    for k in range(2):
        o.rho0[k] = p["rho0"][k]
        o.mu[k] = p["mu"][k]
        o.mass[k] = p["mass"][k]
    return o


def make_piston(m: dict | None) -> OrPiston | None:
    """The oracle's piston struct from a dict with axis, amp, omega, phase
    (equal-length sequences, at most 8) and t_end; None for no motion."""
    if m is None:
        return None
    o = OrPiston()
    o.axis = int(m["axis"])
    o.ncomp = len(m["amp"])
    assert o.ncomp <= 8 and len(m["omega"]) == len(m["phase"]) == o.ncomp
    o.t_end = float(m["t_end"])
    for c in range(o.ncomp):
        o.amp[c], o.omega[c], o.phase[c] = m["amp"][c], m["omega"][c], m["phase"][c]
    return o


def piston_disp(m: dict, t: float) -> float:
    return lib().or_piston_disp(C.byref(make_piston(m)), t)


def piston_vel(m: dict, t: float) -> float:
    return lib().or_piston_vel(C.byref(make_piston(m)), t)


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def W(dim, h, r):
    return lib().or_W(dim, h, r)


def dWdr(dim, h, r):
    return lib().or_dWdr(dim, h, r)


def eos(p: dict, phase: int, rho: float) -> float:
    return lib().or_eos(C.byref(make_params(p)), phase, rho)


def eos_inverse(p: dict, phase: int, pressure: float) -> float:
    return lib().or_eos_inverse(C.byref(make_params(p)), phase, pressure)


def grid_dims(p: dict):
    d = np.zeros(3, np.int32)
    lib().or_grid_dims(C.byref(make_params(p)), _c(d, C.c_int32))
    return tuple(int(v) for v in d)


def cell_ids(p: dict, x: np.ndarray):
    x = np.ascontiguousarray(x, np.float64)
    out = np.empty(len(x), np.int32)
    lib().or_cell_ids(C.byref(make_params(p)), len(x), _d(x), _c(out, C.c_int32))
    return out


def sort_perm(cell: np.ndarray):
    cell = np.ascontiguousarray(cell, np.int32)
    out = np.empty(len(cell), np.int64)
    lib().or_sort_perm(len(cell), _c(cell, C.c_int32), _c(out, C.c_int64))
    return out


def neighbours(p: dict, x: np.ndarray, method: str = "cells"):
    """CSR neighbour sets (start, list), each row ascending."""
    x = np.ascontiguousarray(x, np.float64)
    n = len(x)
    f = lib().or_neighbours_brute if method == "brute" else lib().or_neighbours_cells
    prm = make_params(p)
    start = np.zeros(n + 1, np.int64)
    f(C.byref(prm), n, _d(x), _c(start, C.c_int64), None, 0)
    cap = int(start[n])
    lst = np.zeros(max(cap, 1), np.int32)
    r = f(C.byref(prm), n, _d(x), _c(start, C.c_int64), _c(lst, C.c_int32), cap)
    if r < 0:
        raise RuntimeError(f"oracle neighbour search failed ({r})")
    return start, lst[:cap]


def evaluate(p: dict, x, u, rho, phase, wall, renorm: bool):
    """One rates evaluation; returns dict of rho, P, gradC, T, a, drho."""
    d = int(p["dim"])
    x = np.ascontiguousarray(x, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    phase = np.ascontiguousarray(phase, np.uint8)
    wall = np.ascontiguousarray(wall, np.uint8)
    n = len(x)
    out = dict(rho=np.empty(n), P=np.empty(n), gradC=np.empty((n, d)), T=np.empty((n, d, d)),
               a=np.empty((n, d)), drho=np.empty(n))
    rc = lib().or_eval(C.byref(make_params(p)), n, _d(x), _d(u), _d(rho),
                       _c(phase, C.c_uint8), _c(wall, C.c_uint8), int(bool(renorm)),
                       _d(out["rho"]), _d(out["P"]), _d(out["gradC"]), _d(out["T"]),
                       _d(out["a"]), _d(out["drho"]))
    if rc != 0:
        raise RuntimeError(f"oracle evaluation failed ({rc})")
    return out


def run(p: dict, x, u, rho, phase, wall, dt: float, nsteps: int, first_step: int = 0,
        piston: dict | None = None, t0: float = 0.0):
    """nsteps predictor-corrector steps from time t0; returns new (x, u, rho)
    copies.  Particles with wall == 2 follow the piston motion (if given)."""
    x = np.array(x, np.float64, copy=True, order="C")
    u = np.array(u, np.float64, copy=True, order="C")
    rho = np.array(rho, np.float64, copy=True, order="C")
    phase = np.ascontiguousarray(phase, np.uint8)
    wall = np.ascontiguousarray(wall, np.uint8)
    m = make_piston(piston)
    rc = lib().or_run(C.byref(make_params(p)), len(x), _d(x), _d(u), _d(rho),
                      _c(phase, C.c_uint8), _c(wall, C.c_uint8), dt, first_step, nsteps,
                      C.byref(m) if m is not None else None, t0)
    if rc != 0:
        raise RuntimeError(f"oracle step failed ({rc})")
    return x, u, rho


def diagnostics(p: dict, x, u, phase, wall):
    x = np.ascontiguousarray(x, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    out = np.zeros(12)
    lib().or_diag(C.byref(make_params(p)), len(x), _d(x), _d(u),
                  _c(np.ascontiguousarray(phase, np.uint8), C.c_uint8),
                  _c(np.ascontiguousarray(wall, np.uint8), C.c_uint8), _d(out))
    d = int(p["dim"])
    return dict(mass=out[0], momentum=out[1:1 + d].copy(), e_kin=out[4], e_pot=out[5],
                centroid=out[6:6 + d].copy(), sphericity=out[9], u_max=out[10], n_oil=int(out[11]))


def suggest_dt(p: dict, a=None, wall=None) -> float:
    """Time-step advice for one instance: the smallest of the acoustic bound
    0.25 h / c0, the viscous bound 0.125 h^2 / max(mu / rho0), the capillary
    bound 0.25 sqrt(min(rho0) h^3 / (2 pi alpha_s)) (alpha_s > 0) and the
    body-force bound 0.25 sqrt(h / max |a|) over the fluid particles of `a`
    (when given).  Parity unpinned as a rule: the paper fixes only
    c0 >= 10 u_max (Sec. II-A); the tests check that the advised step is
    stable where a few times larger is not."""
    h = p["h"]
    d = 0.25 * h / p["c0"]
    nu = max(p["mu"][0] / p["rho0"][0], p["mu"][1] / p["rho0"][1])
    if nu > 0:
        d = min(d, 0.125 * h * h / nu)
    if p["alpha_s"] > 0:
        d = min(d, 0.25 * np.sqrt(min(p["rho0"]) * h ** 3 / (2 * np.pi * p["alpha_s"])))
    if a is not None:
        a = np.asarray(a)
        fl = np.ones(len(a), bool) if wall is None else np.asarray(wall) == 0
        amax = np.linalg.norm(a[fl], axis=1).max() if fl.any() else 0.0
        if amax > 0:
            d = min(d, 0.25 * np.sqrt(h / amax))
    return float(d)


def oil_occupancy(p: dict, x, phase, wall):
    """Set of cells (integer tuples) of a grid of spacing d_p = (m_oil /
    rho0_oil)^(1/dim) from box_lo that hold at least one oil particle;
    periodic coordinates are wrapped into the box first."""
    d = int(p["dim"])
    x = np.array(x, np.float64, copy=True)
    per = int(p.get("periodic", 0))
    for k in range(d):
        if (per >> k) & 1:
            L = p["box_hi"][k] - p["box_lo"][k]
            x[:, k] -= L * np.floor((x[:, k] - p["box_lo"][k]) / L)
    dp = (p["mass"][1] / p["rho0"][1]) ** (1.0 / d)
    oil = (np.asarray(phase) == 1) & (np.asarray(wall) == 0)
    c = np.floor((x[oil] - np.array(p["box_lo"][:d])) / dp).astype(np.int64)
    return set(map(tuple, c))


def interface_error(p: dict, xa, xb, phase, wall) -> float:
    """|O_a xor O_b| / |O_b| for the oil occupancies of two states."""
    A, B = oil_occupancy(p, xa, phase, wall), oil_occupancy(p, xb, phase, wall)
    if not B:
        return 0.0 if not A else 1e30
    return len(A ^ B) / len(B)


def set_threads(k: int) -> None:
    lib().or_set_num_threads(int(k))


def num_threads() -> int:
    return int(lib().or_num_threads())
