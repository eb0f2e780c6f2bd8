"""Thin ctypes binding of the C ABI in ``include/sph.h`` (libsph.so).

Argument marshalling only: every step of the particle loop runs in the CUDA
library.  Loading fails loudly when the library is missing; there is no CPU
path.  Arrays are numpy, in the caller's particle order.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsph.so")

SPH_OK = 0
SPH_EFALLBACK = -9
ERRORS = {-1: "SPH_EINVAL", -2: "SPH_ENOMEM", -3: "SPH_ECUDA", -4: "SPH_ENONFINITE",
          -5: "SPH_ECFL", -6: "SPH_EDOMAIN", -7: "SPH_ECAPACITY", -8: "SPH_ETIMEOUT", -9: "SPH_EFALLBACK",
          -10: "SPH_EBOUNDS"}
VISC_DYNAMIC, VISC_KINEMATIC = 0, 1
FIELD = dict(pos=0, vel=1, rho=2, rho_eval=3, pressure=4, acc=5, drho=6, tensor=7, cell=8, order=9)

# entry points declared in include/sph.h and include/sph_surrogate.h
EXPORTS = ["sph_create", "sph_set_state", "sph_build_cells", "sph_eval_rates", "sph_step", "sph_run",
           "sph_sync", "sph_read", "sph_neighbours", "sph_pair_stats", "sph_pair_classes", "sph_diag", "sph_timing_enable",
           "sph_timing_reset", "sph_timing_count", "sph_timing_read", "sph_num_particles",
           "sph_step_index", "sph_num_cells", "sph_list_builds", "sph_destroy", "sph_last_error",
           "sph_cell_sort_noalloc", "sph_create_batch", "sph_set_dt_scales", "sph_run_persistent",
           "sph_set_launch_shape", "sph_get_launch_shape", "sph_autotune", "sph_diag_instances",
           "sph_num_instances", "sph_test_stall_barrier", "sph_mm_bf16", "sph_snapshot", "sph_load_snapshot",
           "sph_surrogate_init", "sph_surrogate_get_weights", "sph_surrogate_predict", "sph_surrogate_advance",
           "sph_surrogate_train_step", "sph_surrogate_run", "sph_create_dev", "sph_set_piston", "sph_get_time",
           "sph_set_time", "sph_suggest_dt", "sph_surrogate_advance_judged", "sph_read_state", "sph_advance_host",
           "sph_oil_occupancy_diff", "sph_surrogate_set_interface_tol", "sph_surrogate_judge_stats",
           "sph_perturb_state", "sph_fp32_peak"]


class SphError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class SphParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("visc_form", C.c_int32), ("renorm_every", C.c_int32),
        ("max_neighbours", C.c_int32), ("rebuild_every", C.c_int32), ("periodic", C.c_int32),
        ("renorm_walls", C.c_int32), ("reserved", C.c_int32),
        ("h", C.c_double), ("c0", C.c_double), ("gamma", C.c_double),
        ("delta", C.c_double), ("alpha_s", C.c_double), ("cell_size", C.c_double), ("skin", C.c_double),
        ("g", C.c_double * 3), ("rho0", C.c_double * 2), ("mu", C.c_double * 2),
        ("mass", C.c_double * 2), ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
    ]


_lib = None


def load(path: str = LIB_PATH):
    """Loads libsph.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libsph.so not found at {path}: run paper_1702_07760_gb300.build.build()")
    L = C.CDLL(path)
    P, vp, dp, u8p = C.POINTER, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_uint8)
    H = C.c_void_p
    L.sph_create.argtypes = [P(SphParams), C.c_int64, dp, dp, dp, u8p, u8p, vp, P(H)]
    L.sph_set_state.argtypes = [H, dp, dp, dp]
    for f in (L.sph_build_cells, L.sph_eval_rates, L.sph_sync, L.sph_timing_reset):
        f.argtypes = [H]
    L.sph_step.argtypes = [H, C.c_double]
    L.sph_run.argtypes = [H, C.c_double, C.c_int64, C.c_int]
    L.sph_read.argtypes = [H, C.c_int, vp, C.c_int64]
    L.sph_read_state.argtypes = [H, dp, dp, dp]
    L.sph_advance_host.argtypes = [H, C.c_double, C.c_int64, dp, dp, dp, dp, dp, dp]
    L.sph_oil_occupancy_diff.argtypes = [H, H, dp]
    L.sph_perturb_state.argtypes = [H, C.c_double, C.c_double, C.c_uint64]
    L.sph_surrogate_set_interface_tol.argtypes = [H, C.c_double]
    L.sph_surrogate_judge_stats.argtypes = [H, dp, dp]
    L.sph_neighbours.argtypes = [H, P(C.c_int64), P(C.c_int32), C.c_int64]
    L.sph_neighbours.restype = C.c_int64
    L.sph_diag.argtypes = [H, dp]
    L.sph_pair_stats.argtypes = [H, P(C.c_int64)]
    L.sph_pair_classes.argtypes = [H, P(C.c_int64)]
    L.sph_timing_enable.argtypes = [H, C.c_int]
    L.sph_timing_count.argtypes = []
    L.sph_timing_read.argtypes = [H, C.c_int, P(C.c_char_p), P(C.c_int64), P(C.c_double)]
    for f in (L.sph_num_particles, L.sph_step_index, L.sph_num_cells, L.sph_list_builds):
        f.argtypes = [H]
        f.restype = C.c_int64
    L.sph_destroy.argtypes = [H]
    L.sph_destroy.restype = None
    L.sph_last_error.restype = C.c_char_p
    L.sph_cell_sort_noalloc.argtypes = [P(SphParams), C.c_int64, vp, vp, vp, vp]
    L.sph_fp32_peak.argtypes = [C.c_int, C.c_int, vp, dp, dp]
    L.sph_create_batch.argtypes = [C.c_int, P(SphParams), P(C.c_int64), dp, dp, dp, u8p, u8p, vp, P(H)]
    L.sph_set_dt_scales.argtypes = [H, dp]
    L.sph_run_persistent.argtypes = [H, C.c_double, C.c_int64, C.c_int]
    L.sph_set_launch_shape.argtypes = [H, C.c_int, C.c_int, C.c_int]
    L.sph_get_launch_shape.argtypes = [H, P(C.c_int), P(C.c_int), P(C.c_int)]
    L.sph_autotune.argtypes = [H, C.c_double, C.c_int, P(C.c_int), P(C.c_int), P(C.c_int), dp]
    L.sph_diag_instances.argtypes = [H, dp]
    L.sph_num_instances.argtypes = [H]
    L.sph_test_stall_barrier.argtypes = [H]
    L.sph_mm_bf16.argtypes = [vp, C.c_int, vp, C.c_int, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                              vp, vp]
    L.sph_snapshot.argtypes = [H, vp, vp, vp]
    L.sph_load_snapshot.argtypes = [H, vp, vp, vp]
    L.sph_surrogate_init.argtypes = [H, dp, C.c_int64, dp, C.c_int64]
    L.sph_surrogate_get_weights.argtypes = [H, dp, C.c_int64]
    L.sph_surrogate_predict.argtypes = [H, dp, C.c_int64]
    L.sph_surrogate_advance.argtypes = [H, C.c_int]
    L.sph_surrogate_train_step.argtypes = [H, vp, vp, vp, C.c_double, C.c_int, dp, dp, C.c_int64]
    L.sph_surrogate_run.argtypes = [H, C.c_double, C.c_int, C.c_int64, C.c_int, C.c_double, C.c_double,
                                    P(C.c_int64), P(C.c_int64), dp]
    L.sph_num_instances.restype = C.c_int64
    L.sph_create_dev.argtypes = [P(SphParams), C.c_int64, vp, vp, vp, vp, vp, vp, P(H)]
    L.sph_set_piston.argtypes = [H, C.c_int, C.c_int, dp, dp, dp, C.c_double]
    L.sph_get_time.argtypes = [H, dp]
    L.sph_set_time.argtypes = [H, C.c_double]
    L.sph_suggest_dt.argtypes = [H, dp]
    L.sph_surrogate_advance_judged.argtypes = [H, C.c_double, C.c_int, C.c_double, C.c_double, dp]
    _lib = L
    return L


def make_params(p: dict) -> SphParams:
    s = SphParams()
    s.dim = int(p["dim"])
    s.visc_form = int(p.get("visc_form", 0))
    s.renorm_every = int(p.get("renorm_every", 1))
    s.max_neighbours = int(p.get("max_neighbours", 0))
    s.rebuild_every = int(p.get("rebuild_every", 0))
    s.periodic = int(p.get("periodic", 0))
    s.renorm_walls = int(p.get("renorm_walls", 1))
    s.h, s.c0, s.gamma = p["h"], p["c0"], p.get("gamma", 7.0)
    s.delta, s.alpha_s, s.cell_size, s.skin = p["delta"], p["alpha_s"], p["cell_size"], p["skin"]
    for k in range(3):
        s.g[k], s.box_lo[k], s.box_hi[k] = p["g"][k], p["box_lo"][k], p["box_hi"][k]
    for k in range(2):
        s.rho0[k], s.mu[k], s.mass[k] = p["rho0"][k], p["mu"][k], p["mass"][k]
    return s


def _check(rc: int):
    if rc != SPH_OK:
        raise SphError(rc, load().sph_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def cell_sort_noalloc(params: dict, n: int, x_dev: int, cell_dev: int, order_dev: int, stream: int = 0):
    """Allocation-free cell sort on device arrays given by address (see
    sph_cell_sort_noalloc in include/sph.h)."""
    p = make_params(params)
    _check(load().sph_cell_sort_noalloc(C.byref(p), int(n), C.c_void_p(x_dev), C.c_void_p(cell_dev),
                                        C.c_void_p(order_dev), C.c_void_p(stream)))


def fp32_peak(blocks_per_sm: int = 8, iters: int = 4096, stream: int = 0):
    """(TFLOP/s, ms): FP32 FMA throughput of the current device (see
    sph_fp32_peak in include/sph.h)."""
    t, m = C.c_double(), C.c_double()
    _check(load().sph_fp32_peak(int(blocks_per_sm), int(iters), C.c_void_p(stream), C.byref(t), C.byref(m)))
    return t.value, m.value


def mm_bf16(a_ptr: int, lda: int, b_ptr: int, ldb: int, c_ptr: int, ldc: int, M: int, N: int, K: int,
            k_split: int = 0, accumulate: bool = False, stream: int = 0, err_ptr: int = 0):
    """C = A B^T on the tensor cores for device arrays given by address (see
    sph_mm_bf16 in include/sph_surrogate.h)."""
    _check(load().sph_mm_bf16(C.c_void_p(a_ptr), lda, C.c_void_p(b_ptr), ldb, C.c_void_p(c_ptr), ldc, M, N, K,
                              k_split, int(bool(accumulate)), C.c_void_p(stream), C.c_void_p(err_ptr)))


class Simulation:
    """One two-phase SPH simulation resident on the GPU."""

    def __init__(self, params: dict, x, u, rho, phase, wall, stream: int | None = None):
        L = load()
        self.params = dict(params)
        self.dim = int(params["dim"])
        x = np.ascontiguousarray(x, np.float64)
        u = np.ascontiguousarray(u, np.float64)
        rho = np.ascontiguousarray(rho, np.float64)
        phase = np.ascontiguousarray(phase, np.uint8)
        wall = np.ascontiguousarray(wall, np.uint8)
        self.n = len(x)
        self._p = make_params(params)
        h = C.c_void_p()
        _check(L.sph_create(C.byref(self._p), self.n, _dp(x), _dp(u), _dp(rho),
                            phase.ctypes.data_as(C.POINTER(C.c_uint8)),
                            wall.ctypes.data_as(C.POINTER(C.c_uint8)),
                            C.c_void_p(stream or 0), C.byref(h)))
        self._h = h

    @classmethod
    def from_workload(cls, w, stream=None):
        return cls(w.params, w.x, w.u, w.rho, w.phase, w.wall, stream)

    @classmethod
    def from_device(cls, params: dict, n: int, x_ptr: int, u_ptr: int, rho_ptr: int, phase_ptr: int,
                    wall_ptr: int, stream: int | None = None) -> "Simulation":
        """sph_create_dev: the initial state from device arrays given by
        address (x, u: n*dim float64; rho: n float64; phase, wall: n uint8)."""
        self = cls.__new__(cls)
        self.params = dict(params)
        self.dim = int(params["dim"])
        self.n = int(n)
        self._p = make_params(params)
        self._h = None
        h = C.c_void_p()
        _check(load().sph_create_dev(C.byref(self._p), self.n, C.c_void_p(x_ptr), C.c_void_p(u_ptr),
                                     C.c_void_p(rho_ptr), C.c_void_p(phase_ptr), C.c_void_p(wall_ptr),
                                     C.c_void_p(stream or 0), C.byref(h)))
        self._h = h
        return self

    def set_piston(self, axis: int, amp, omega, phase, t_end: float):
        """Prescribed motion of the particles with wall == 2 (sph_set_piston)."""
        a = np.ascontiguousarray(amp, np.float64)
        w = np.ascontiguousarray(omega, np.float64)
        f = np.ascontiguousarray(phase, np.float64)
        if not (len(a) == len(w) == len(f)):
            raise ValueError("amp, omega and phase must have equal lengths")
        _check(load().sph_set_piston(self._h, int(axis), len(a), _dp(a), _dp(w), _dp(f), float(t_end)))

    @property
    def time(self) -> float:
        t = C.c_double()
        _check(load().sph_get_time(self._h, C.byref(t)))
        return t.value

    def set_time(self, t: float):
        _check(load().sph_set_time(self._h, float(t)))

    def suggest_dt(self) -> float:
        dt = C.c_double()
        _check(load().sph_suggest_dt(self._h, C.byref(dt)))
        return dt.value

    @classmethod
    def batch(cls, workloads, stream: int | None = None) -> "Simulation":
        """One handle over independent instances (sph_create_batch): the
        workloads' particles one after another, each in its own frame."""
        L = load()
        self = cls.__new__(cls)
        k = len(workloads)
        self.params = dict(workloads[0].params)
        self.dim = int(self.params["dim"])
        ps = (SphParams * k)(*[make_params(w.params) for w in workloads])
        counts = np.array([w.n for w in workloads], np.int64)
        x = np.ascontiguousarray(np.concatenate([w.x for w in workloads]), np.float64)
        u = np.ascontiguousarray(np.concatenate([w.u for w in workloads]), np.float64)
        rho = np.ascontiguousarray(np.concatenate([w.rho for w in workloads]), np.float64)
        phase = np.ascontiguousarray(np.concatenate([w.phase for w in workloads]), np.uint8)
        wall = np.ascontiguousarray(np.concatenate([w.wall for w in workloads]), np.uint8)
        self.n = len(x)
        self._p = ps
        self.first = np.concatenate([[0], np.cumsum(counts)])
        h = C.c_void_p()
        self._h = None
        _check(L.sph_create_batch(k, ps, counts.ctypes.data_as(C.POINTER(C.c_int64)), _dp(x), _dp(u),
                                  _dp(rho), phase.ctypes.data_as(C.POINTER(C.c_uint8)),
                                  wall.ctypes.data_as(C.POINTER(C.c_uint8)), C.c_void_p(stream or 0),
                                  C.byref(h)))
        self._h = h
        return self

    @property
    def num_instances(self) -> int:
        return int(load().sph_num_instances(self._h))

    def set_dt_scales(self, scales):
        sc = np.ascontiguousarray(scales, np.float64)
        if len(sc) != self.num_instances:
            raise ValueError("one scale per instance")
        _check(load().sph_set_dt_scales(self._h, _dp(sc)))

    # -- stepping ---------------------------------------------------------
    def set_state(self, x, u, rho):
        x = np.ascontiguousarray(x, np.float64)
        u = np.ascontiguousarray(u, np.float64)
        rho = np.ascontiguousarray(rho, np.float64)
        _check(load().sph_set_state(self._h, _dp(x), _dp(u), _dp(rho)))

    def build_cells(self):
        _check(load().sph_build_cells(self._h))

    def eval_rates(self):
        _check(load().sph_eval_rates(self._h))

    def step(self, dt: float):
        _check(load().sph_step(self._h, dt))

    def run(self, dt: float, nsteps: int, graph: bool = True):
        _check(load().sph_run(self._h, dt, int(nsteps), int(bool(graph))))

    def run_persistent(self, dt: float, nsteps: int, graph: bool = True):
        """nsteps steps in one cooperative launch (sph_run_persistent)."""
        _check(load().sph_run_persistent(self._h, dt, int(nsteps), int(bool(graph))))

    def set_launch_shape(self, block: int, grid_blocks: int = 0, dynamic_chunks: bool = True):
        _check(load().sph_set_launch_shape(self._h, int(block), int(grid_blocks), int(bool(dynamic_chunks))))

    def launch_shape(self):
        """(block, grid blocks, dynamic chunks) of the persistent launch on this device."""
        b, g, d = C.c_int(), C.c_int(), C.c_int()
        _check(load().sph_get_launch_shape(self._h, C.byref(b), C.byref(g), C.byref(d)))
        return b.value, g.value, bool(d.value)

    def autotune(self, dt: float, trial_steps: int = 20):
        """Fastest persistent launch shape: (block, grid blocks, dynamic chunks, ms per step)."""
        b, g, d, ms = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        _check(load().sph_autotune(self._h, dt, int(trial_steps), C.byref(b), C.byref(g), C.byref(d),
                                   C.byref(ms)))
        return b.value, g.value, bool(d.value), ms.value

    def test_stall_barrier(self):
        """Makes the next run_persistent time out at its first barrier (test support)."""
        _check(load().sph_test_stall_barrier(self._h))

    def sync(self):
        _check(load().sph_sync(self._h))

    # -- snapshots and the learned surrogate ------------------------------
    def snapshot_to(self, x_ptr: int, u_ptr: int, rho_ptr: int):
        """Queues a copy of the state (original order) into device arrays given by address."""
        _check(load().sph_snapshot(self._h, C.c_void_p(x_ptr), C.c_void_p(u_ptr), C.c_void_p(rho_ptr)))

    def load_snapshot(self, x_ptr: int, u_ptr: int, rho_ptr: int):
        _check(load().sph_load_snapshot(self._h, C.c_void_p(x_ptr), C.c_void_p(u_ptr), C.c_void_p(rho_ptr)))

    def surrogate_init(self, weights, norm):
        w = np.ascontiguousarray(weights, np.float64)
        nm = np.ascontiguousarray(norm, np.float64)
        _check(load().sph_surrogate_init(self._h, _dp(w), len(w), _dp(nm), len(nm)))
        self._nweights = len(w)

    def surrogate_weights(self) -> np.ndarray:
        w = np.zeros(self._nweights)
        _check(load().sph_surrogate_get_weights(self._h, _dp(w), len(w)))
        return w

    def surrogate_predict(self) -> np.ndarray:
        """(n, 2 dim + 1) increments dx, du, drho in original order."""
        out = np.zeros((self.n, 2 * self.dim + 1))
        _check(load().sph_surrogate_predict(self._h, _dp(out), out.nbytes))
        return out

    def surrogate_advance(self, k_steps: int):
        _check(load().sph_surrogate_advance(self._h, int(k_steps)))

    def surrogate_train_step(self, x1_ptr: int, u1_ptr: int, rho1_ptr: int, lr: float = 1e-3,
                             update: bool = True, want_grad: bool = False):
        """(loss, gradient or None) of one training step towards the state after k steps."""
        loss = C.c_double()
        g = np.zeros(self._nweights) if want_grad else None
        _check(load().sph_surrogate_train_step(self._h, C.c_void_p(x1_ptr), C.c_void_p(u1_ptr),
                                               C.c_void_p(rho1_ptr), float(lr), int(bool(update)), C.byref(loss),
                                               _dp(g) if want_grad else None, self._nweights if want_grad else 0))
        return loss.value, g

    def surrogate_run(self, dt: float, k_steps: int, n_macro: int, judge_every: int, tol: float, d_ref: float):
        """(judged, rejected, largest judged centroid error / d_ref)."""
        a, b, e = C.c_int64(), C.c_int64(), C.c_double()
        _check(load().sph_surrogate_run(self._h, float(dt), int(k_steps), int(n_macro), int(judge_every),
                                        float(tol), float(d_ref), C.byref(a), C.byref(b), C.byref(e)))
        return a.value, b.value, e.value

    def perturb(self, sigma_u: float, sigma_rho: float, seed: int):
        """Gaussian noise on the fluid velocities and densities (sph_perturb_state)."""
        _check(load().sph_perturb_state(self._h, float(sigma_u), float(sigma_rho), int(seed) & (2 ** 64 - 1)))

    def interface_error(self, plain: "Simulation") -> float:
        """Oil occupancy difference against another handle (sph_oil_occupancy_diff)."""
        e = C.c_double()
        _check(load().sph_oil_occupancy_diff(self._h, plain._h, C.byref(e)))
        return e.value

    def surrogate_set_interface_tol(self, tol: float):
        _check(load().sph_surrogate_set_interface_tol(self._h, float(tol)))

    def surrogate_judge_stats(self):
        """(largest centroid error / d_ref, largest interface error) of the last judged run."""
        a, b = C.c_double(), C.c_double()
        _check(load().sph_surrogate_judge_stats(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def surrogate_advance_judged(self, dt: float, k_steps: int, tol: float, d_ref: float):
        """One judged macro-step (sph_surrogate_advance_judged): returns
        (accepted, centroid error / d_ref); the state is the plain result."""
        e = C.c_double()
        rc = load().sph_surrogate_advance_judged(self._h, float(dt), int(k_steps), float(tol), float(d_ref),
                                                 C.byref(e))
        if rc not in (SPH_OK, SPH_EFALLBACK):
            _check(rc)
        return rc == SPH_OK, e.value

    # -- output -----------------------------------------------------------
    def read_state(self, x: np.ndarray, u: np.ndarray, rho: np.ndarray):
        """x, u, rho into the given C-contiguous float64 arrays (e.g. pinned)
        with one call (sph_read_state)."""
        n, d = self.n, self.dim
        for a, shape in ((x, (n, d)), (u, (n, d)), (rho, (n,))):
            if a.shape != shape or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"expected a C-contiguous float64 array of shape {shape}")
        _check(load().sph_read_state(self._h, _dp(x), _dp(u), _dp(rho)))

    def advance_host(self, dt: float, nsteps: int, x: np.ndarray, u: np.ndarray, rho: np.ndarray,
                     out=None):
        """Loads (x, u, rho), runs nsteps graph-replayed steps and writes the
        result into `out` = (x, u, rho) arrays (default: the inputs) with one
        call and one wait (sph_advance_host)."""
        n, d = self.n, self.dim
        xo, uo, ro = (x, u, rho) if out is None else out
        for a, shape in ((x, (n, d)), (u, (n, d)), (rho, (n,)), (xo, (n, d)), (uo, (n, d)), (ro, (n,))):
            if a.shape != shape or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"expected a C-contiguous float64 array of shape {shape}")
        _check(load().sph_advance_host(self._h, float(dt), int(nsteps), _dp(x), _dp(u), _dp(rho),
                                       _dp(xo), _dp(uo), _dp(ro)))

    def read(self, field: str, out: np.ndarray | None = None) -> np.ndarray:
        """Copies a field in original particle order into `out` (a C-contiguous
        array of the field's shape and type, e.g. in pinned host memory) or a
        new array."""
        n, d = self.n, self.dim
        shapes = dict(pos=(n, d), vel=(n, d), acc=(n, d), tensor=(n, d, d))
        shape = shapes.get(field, (n,))
        dtype = np.int32 if field in ("cell", "order") else np.float64
        if out is None:
            out = np.empty(shape, dtype)
        elif out.shape != shape or out.dtype != dtype or not out.flags["C_CONTIGUOUS"]:
            raise ValueError(f"out must be a C-contiguous {dtype.__name__} array of shape {shape}")
        _check(load().sph_read(self._h, FIELD[field], out.ctypes.data_as(C.c_void_p), out.nbytes))
        return out

    def neighbours(self):
        L = load()
        start = np.zeros(self.n + 1, np.int64)
        L.sph_neighbours(self._h, start.ctypes.data_as(C.POINTER(C.c_int64)), None, 0)
        cap = int(start[-1])
        lst = np.zeros(max(cap, 1), np.int32)
        r = L.sph_neighbours(self._h, start.ctypes.data_as(C.POINTER(C.c_int64)),
                             lst.ctypes.data_as(C.POINTER(C.c_int32)), cap)
        if r < 0:
            _check(int(r))
        return start, lst[:cap]

    def pair_stats(self):
        """(ordered neighbour pairs, of which across phases) at the current positions."""
        out = np.zeros(2, np.int64)
        _check(load().sph_pair_stats(self._h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return int(out[0]), int(out[1])

    def pair_classes(self):
        """(ordered neighbour pairs, across phases, between two static boundary
        particles, of a static boundary particle with another) at the current
        positions (sph_pair_classes)."""
        out = np.zeros(4, np.int64)
        _check(load().sph_pair_classes(self._h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return tuple(int(v) for v in out)

    @staticmethod
    def _diag_dict(out, d):
        return dict(mass=out[0], momentum=out[1:1 + d].copy(), e_kin=out[4], e_pot=out[5],
                    centroid=out[6:6 + d].copy(), sphericity=out[9], u_max=out[10], n_oil=int(out[11]))

    def diagnostics(self) -> dict:
        out = np.zeros(12)
        _check(load().sph_diag(self._h, _dp(out)))
        return self._diag_dict(out, self.dim)

    def diagnostics_instances(self) -> list:
        """diagnostics() of every instance of a batch, positions in each instance's frame."""
        k = self.num_instances
        out = np.zeros(12 * k)
        _check(load().sph_diag_instances(self._h, _dp(out)))
        return [self._diag_dict(out[12 * q:12 * q + 12], self.dim) for q in range(k)]

    # -- timing -----------------------------------------------------------
    def timing(self, enable: bool):
        _check(load().sph_timing_enable(self._h, int(bool(enable))))

    def timing_reset(self):
        _check(load().sph_timing_reset(self._h))

    def timing_read(self) -> dict:
        L = load()
        res = {}
        for k in range(L.sph_timing_count()):
            name, cnt, ms = C.c_char_p(), C.c_int64(), C.c_double()
            _check(L.sph_timing_read(self._h, k, C.byref(name), C.byref(cnt), C.byref(ms)))
            res[name.value.decode()] = (int(cnt.value), float(ms.value))
        return res

    @property
    def step_index(self) -> int:
        return int(load().sph_step_index(self._h))

    @property
    def list_builds(self) -> int:
        r = int(load().sph_list_builds(self._h))
        if r < 0:
            _check(r)
        return r

    @property
    def num_cells(self) -> int:
        return int(load().sph_num_cells(self._h))

    def close(self):
        if getattr(self, "_h", None):
            load().sph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
