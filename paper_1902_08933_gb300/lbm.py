"""ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every computation runs in liblbm.so's CUDA kernels; this module converts
Python arguments to the C types and status codes to exceptions. If the library
is missing the first call raises: there is no CPU fallback.

Functions carry the C names (``lbm_create``, ``lbm_init``, ``lbm_step``,
``lbm_get_fields``, ...). ``Simulation`` is a small convenience wrapper over
them for the tests and the benchmark.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

# enums of include/lbm.h
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_ESTATE, LBM_EIO = range(8)
LBM_BC_PERIODIC, LBM_BC_BOUNCEBACK = 0, 1
LBM_IM, LBM_QIM = 0, 1
LBM_P_MODIFIED_PRINTED, LBM_P_MODIFIED_LITERAL, LBM_P_PREVIOUS = 0, 1, 2
LBM_FS_MU_GRADPHI, LBM_FS_PHI_GRADMU = 0, 1
LBM_VISC_INV_LINEAR, LBM_VISC_STEP = 0, 1
LBM_F64, LBM_F32, LBM_F32_G16, LBM_F32_H16, LBM_F32_C, LBM_F32_CC = 0, 1, 2, 3, 4, 5
LBM_PIPELINE_AUTO, LBM_PIPELINE_PLAIN, LBM_PIPELINE_ASYNC, LBM_PIPELINE_TMA, LBM_PIPELINE_PAIRS = 0, 1, 2, 3, 4
LBM_PIPELINE_BATCHED = 5
LBM_PIPELINE_PERSISTENT = 6
VARIANTS = {0: "plain", 1: "async", 2: "tma", 3: "pairs", 4: "batched"}
FIELDS = ("phi", "ux", "uy", "p", "rho", "mu", "P")
FIELDS3 = FIELDS + ("uz",)          # D3Q15 lattices (nz >= 2) also have uz
FIELD_BITS = {name: 1 << k for k, name in enumerate(FIELDS3)}
FORMS = {"f64": LBM_F64, "f32": LBM_F32, "f32_g16": LBM_F32_G16, "f32_h16": LBM_F32_H16,
         "f32_c": LBM_F32_C, "f32_cc": LBM_F32_CC}
# bytes moved per lattice update (every population read and written once, plus phi*u, p)
BYTES_PER_LUP = {"f64": 336, "f32": 168, "f32_g16": 140, "f32_h16": 108, "f32_c": 176, "f32_cc": 176}

_STATUS = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_ENONFINITE",
           5: "LBM_ETIMEOUT", 6: "LBM_ESTATE", 7: "LBM_EIO"}


class LbmError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class lbm_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("bc_y", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("pressure_scheme", ctypes.c_int32),
                ("surface_force", ctypes.c_int32), ("viscosity_model", ctypes.c_int32),
                ("nz", ctypes.c_int32)] + [
        (n, ctypes.c_double) for n in ("rho_A", "rho_B", "nu_A", "nu_B", "sigma", "W", "tau_h",
                                       "mobility", "force_x", "force_y", "gravity")]


class lbm_diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "sum_phi", "sum_rho", "kinetic_energy", "max_u", "centroid_A_x", "centroid_A_y",
        "centroid_B_x", "centroid_B_y", "mass_A", "mass_B", "P_bulk_A", "P_bulk_B",
        "n_bulk_A", "n_bulk_B")] + [("nonfinite", ctypes.c_int32), ("reserved", ctypes.c_int32),
                                     ("time", ctypes.c_int64)]


class lbm_monitor(ctypes.Structure):
    _fields_ = [("sum_phi", ctypes.c_double), ("kinetic_energy", ctypes.c_double),
                ("max_u", ctypes.c_double), ("nonfinite", ctypes.c_int32),
                ("device_status", ctypes.c_int32), ("time", ctypes.c_int64)]


class lbm_launch_shape(ctypes.Structure):
    _fields_ = [("pipeline", ctypes.c_int32), ("tile_x", ctypes.c_int32), ("rows", ctypes.c_int32),
                ("trials", ctypes.c_int32), ("ms_per_step", ctypes.c_double),
                ("default_ms_per_step", ctypes.c_double)]


class lbm_sp_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("bc_y", ctypes.c_int32),
                ("model", ctypes.c_int32), ("nu", ctypes.c_double), ("xi", ctypes.c_double),
                ("force_x", ctypes.c_double), ("force_y", ctypes.c_double), ("scheme", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("drag_lin", ctypes.c_double), ("drag_quad", ctypes.c_double),
                ("p0", ctypes.c_double)]


_lock = threading.Lock()
_lib = None
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)

# (name, restype, argtypes) of every entry point declared in include/lbm.h
SIGNATURES = [
    ("lbm_validate_params", ctypes.c_int, [ctypes.POINTER(lbm_params)]),
    ("lbm_create", ctypes.c_int, [ctypes.POINTER(lbm_params), ctypes.c_int, ctypes.c_int, _VP,
                                  ctypes.POINTER(_VP)]),
    ("lbm_init", ctypes.c_int, [_VP, ctypes.c_int, _DP]),
    ("lbm_init_device", ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    ("lbm_step", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lbm_set_monitor", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lbm_read_monitor", ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(lbm_monitor)]),
    ("lbm_read_monitor_async", ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    ("lbm_step_monitored", ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    ("lbm_step_monitored_all", ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    ("lbm_get_fields", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_uint, _DP]),
    ("lbm_get_fields_device", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_uint, _VP]),
    ("lbm_diagnostics", ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(lbm_diag)]),
    ("lbm_get_populations", ctypes.c_int, [_VP, ctypes.c_int, _DP, _DP]),
    ("lbm_save", ctypes.c_int, [_VP, ctypes.c_char_p]),
    ("lbm_load", ctypes.c_int, [_VP, ctypes.c_char_p]),
    ("lbm_set_launch", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    ("lbm_set_pipeline", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lbm_set_graphs", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lbm_launch_info", ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("lbm_autotune", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("lbm_autotune_shape", ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(lbm_launch_shape)]),
    ("lbm_row_bytes", ctypes.c_size_t, [_VP, ctypes.c_int]),
    ("lbm_measure_fp64_fma", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    ("lbm_pack_rows", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_size_t]),
    ("lbm_unpack_rows", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_size_t]),
    ("lbm_launches_per_step", ctypes.c_int, [_VP]),
    ("lbm_step_launch_count", ctypes.c_longlong, [_VP]),
    ("lbm_time", ctypes.c_int64, [_VP, ctypes.c_int]),
    ("lbm_reduce_fields_noalloc", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    ("lbm_inject_wait_timeout", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lbm_inject_batched_wait_timeout", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lbm_sync", ctypes.c_int, [_VP]),
    ("lbm_last_error", ctypes.c_char_p, [_VP]),
    ("lbm_destroy", None, [_VP]),
    ("lbm_sp_create", ctypes.c_int, [ctypes.POINTER(lbm_sp_params), ctypes.c_int, _VP,
                                     ctypes.POINTER(_VP)]),
    ("lbm_sp_init", ctypes.c_int, [_VP, _DP]),
    ("lbm_sp_step", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lbm_sp_get_fields", ctypes.c_int, [_VP, ctypes.c_uint, _DP]),
    ("lbm_sp_get_populations", ctypes.c_int, [_VP, _DP]),
    ("lbm_sp_last_error", ctypes.c_char_p, [_VP]),
    ("lbm_sp_destroy", None, [_VP]),
]


def library():
    """Load liblbm.so (raises if it was not built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("liblbm.so not found at %s; build it with "
                                   "`python -m paper_1902_08933_gb300.build`" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(st, ctx=None):
    if st != LBM_OK:
        msg = library().lbm_last_error(ctx).decode() if ctx else ""
        raise LbmError(st, msg)


def make_params(cfg: dict) -> lbm_params:
    """lbm_params from a workload dictionary (keys of workloads.PARAM_KEYS)."""
    p = lbm_params()
    p.nx, p.ny = int(cfg["nx"]), int(cfg["ny"])
    p.bc_y = int(cfg.get("walls_y", 0))
    p.variant = int(cfg.get("qim", 1))
    p.pressure_scheme = int(cfg.get("pressure", 0))
    p.surface_force = int(cfg.get("surface_force", 0))
    p.viscosity_model = int(cfg.get("viscosity", 0))
    p.nz = int(cfg.get("nz", 0))
    for k, src in (("rho_A", "rho_A"), ("rho_B", "rho_B"), ("nu_A", "nu_A"), ("nu_B", "nu_B"),
                   ("sigma", "sigma"), ("W", "W"), ("tau_h", "tau_h"), ("mobility", "M"),
                   ("force_x", "force_x"), ("force_y", "force_y"), ("gravity", "gravity")):
        setattr(p, k, float(cfg.get(src, 0.0)))
    return p


# ---- thin wrappers with the C names ---------------------------------------------
def lbm_validate_params(p: lbm_params) -> int:
    return library().lbm_validate_params(ctypes.byref(p))


def lbm_create(params, precision=LBM_F64, stream=None):
    arr = (lbm_params * len(params))(*params)
    out = _VP()
    st = library().lbm_create(arr, len(params), int(precision), _VP(stream or 0), ctypes.byref(out))
    _check(st)
    return out.value


def lbm_init(ctx, instance, phi0: np.ndarray):
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    _check(library().lbm_init(ctx, instance, phi0.ctypes.data_as(_DP)), ctx)


def lbm_init_device(ctx, instance, dev_ptr: int):
    _check(library().lbm_init_device(ctx, instance, _VP(dev_ptr)), ctx)


def lbm_step(ctx, nsteps: int):
    _check(library().lbm_step(ctx, int(nsteps)), ctx)


def lbm_set_monitor(ctx, enable: bool):
    _check(library().lbm_set_monitor(ctx, 1 if enable else 0), ctx)


def lbm_read_monitor(ctx, instance: int) -> dict:
    """Monitor record of the last monitored step; 'status' is LBM_OK or LBM_ENONFINITE."""
    m = lbm_monitor()
    st = library().lbm_read_monitor(ctx, int(instance), ctypes.byref(m))
    if st not in (LBM_OK, LBM_ENONFINITE):
        _check(st, ctx)
    return {"sum_phi": m.sum_phi, "kinetic_energy": m.kinetic_energy, "max_u": m.max_u,
            "time": m.time, "status": st}


def lbm_step_monitored(ctx, nsteps: int, host_records_ptr: int):
    """lbm_step whose monitored last step writes the records (one lbm_monitor per
    instance) into pinned host memory at host_records_ptr, from the GPU."""
    _check(library().lbm_step_monitored(ctx, int(nsteps), _VP(host_records_ptr)), ctx)


def lbm_step_monitored_all(ctx, nsteps: int, host_records_ptr: int):
    """lbm_step writing the record of every step (nsteps x instances lbm_monitor
    records, [step][instance]) into pinned host memory at host_records_ptr, from
    the GPU."""
    _check(library().lbm_step_monitored_all(ctx, int(nsteps), _VP(host_records_ptr)), ctx)


def lbm_read_monitor_async(ctx, instance: int, host_record_ptr: int):
    """Queues the copy of the record into caller memory at host_record_ptr (an
    lbm_monitor's address, ideally pinned); read it after the stream passes."""
    _check(library().lbm_read_monitor_async(ctx, int(instance), _VP(host_record_ptr)), ctx)


def lbm_get_fields(ctx, instance, mask: int, out: np.ndarray):
    assert out.dtype == np.float64 and out.flags.c_contiguous
    _check(library().lbm_get_fields(ctx, instance, mask, out.ctypes.data_as(_DP)), ctx)


def lbm_get_fields_device(ctx, instance, mask: int, dev_ptr: int):
    _check(library().lbm_get_fields_device(ctx, instance, mask, _VP(dev_ptr)), ctx)


def lbm_diagnostics(ctx, instance) -> dict:
    d = lbm_diag()
    st = library().lbm_diagnostics(ctx, instance, ctypes.byref(d))
    out = {k: getattr(d, k) for k, _ in lbm_diag._fields_ if k != "reserved"}
    if st not in (LBM_OK, LBM_ENONFINITE):
        _check(st, ctx)
    out["status"] = st
    return out


def lbm_get_populations(ctx, instance, nx, ny, nz=0):
    """h, g in FP64: (9, ny, nx) on D2Q9, (15, nz, ny, nx) on D3Q15 (nz >= 2)."""
    shape = (15, nz, ny, nx) if nz >= 2 else (9, ny, nx)
    h = np.zeros(shape)
    g = np.zeros(shape)
    _check(library().lbm_get_populations(ctx, instance, h.ctypes.data_as(_DP), g.ctypes.data_as(_DP)), ctx)
    return h, g


def lbm_save(ctx, path: str):
    _check(library().lbm_save(ctx, path.encode()), ctx)


def lbm_load(ctx, path: str):
    _check(library().lbm_load(ctx, path.encode()), ctx)


def lbm_set_launch(ctx, tile_x: int, rows: int):
    _check(library().lbm_set_launch(ctx, int(tile_x), int(rows)), ctx)


def lbm_set_pipeline(ctx, mode: int):
    _check(library().lbm_set_pipeline(ctx, int(mode)), ctx)


def lbm_set_graphs(ctx, enable: bool):
    _check(library().lbm_set_graphs(ctx, 1 if enable else 0), ctx)


def lbm_launch_info(ctx, index: int) -> dict:
    t, b, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(library().lbm_launch_info(ctx, int(index), ctypes.byref(t), ctypes.byref(b), ctypes.byref(m)), ctx)
    return {"tile_x": t.value, "blocks": b.value, "variant": VARIANTS.get(m.value, m.value)}


def lbm_autotune(ctx):
    t, r = ctypes.c_int(), ctypes.c_int()
    _check(library().lbm_autotune(ctx, ctypes.byref(t), ctypes.byref(r)), ctx)
    return t.value, r.value


def lbm_measure_fp64_fma(stream=None) -> float:
    """Measured FP64 FMA throughput of the current GPU, TFLOP/s."""
    t = ctypes.c_double()
    _check(library().lbm_measure_fp64_fma(_VP(stream or 0), ctypes.byref(t)))
    return t.value


def lbm_row_bytes(ctx, instance: int) -> int:
    """Bytes of state one row of an instance takes (0 if not applicable)."""
    return int(library().lbm_row_bytes(ctx, int(instance)))


def lbm_pack_rows(ctx, instance: int, y0: int, nrows: int, dev_ptr: int, nbytes: int):
    """Queues the copy of rows [y0, y0 + nrows) of the instance's state into
    caller device memory at dev_ptr (nbytes available)."""
    _check(library().lbm_pack_rows(ctx, int(instance), int(y0), int(nrows), _VP(dev_ptr), int(nbytes)), ctx)


def lbm_unpack_rows(ctx, instance: int, y0: int, nrows: int, dev_ptr: int, nbytes: int):
    """Queues the copy of rows [y0, y0 + nrows) of the instance's state from
    caller device memory at dev_ptr."""
    _check(library().lbm_unpack_rows(ctx, int(instance), int(y0), int(nrows), _VP(dev_ptr), int(nbytes)), ctx)


LBM_TUNE_NO_CACHE = 1
PIPELINES = {0: "auto", 1: "plain", 2: "async", 3: "tma", 4: "pairs", 5: "batched", 6: "persistent"}


def lbm_autotune_shape(ctx, flags: int = 0) -> dict:
    """Runs (or takes from the cache) the autotuner; returns the chosen shape."""
    r = lbm_launch_shape()
    _check(library().lbm_autotune_shape(ctx, int(flags), ctypes.byref(r)), ctx)
    return {"pipeline": PIPELINES.get(r.pipeline, r.pipeline), "tile_x": r.tile_x, "rows": r.rows,
            "trials": r.trials, "ms_per_step": r.ms_per_step,
            "default_ms_per_step": r.default_ms_per_step}


def lbm_launches_per_step(ctx) -> int:
    return library().lbm_launches_per_step(ctx)


def lbm_step_launch_count(ctx) -> int:
    """Kernel launches the context's lbm_step calls have queued so far."""
    return library().lbm_step_launch_count(ctx)


def lbm_time(ctx, instance) -> int:
    return library().lbm_time(ctx, instance)


def lbm_reduce_fields_noalloc(fields_dev_ptr: int, nx: int, ny: int, stream, out_dev_ptr: int) -> int:
    """Returns the status code (allocation-free FP64 reduction of caller fields)."""
    return library().lbm_reduce_fields_noalloc(_VP(fields_dev_ptr), int(nx), int(ny),
                                               _VP(stream or 0), _VP(out_dev_ptr))


def lbm_inject_wait_timeout(ctx, rounds: int):
    _check(library().lbm_inject_wait_timeout(ctx, int(rounds)), ctx)


def lbm_inject_batched_wait_timeout(ctx, rounds: int):
    _check(library().lbm_inject_batched_wait_timeout(ctx, int(rounds)), ctx)


def lbm_sync(ctx):
    _check(library().lbm_sync(ctx), ctx)


def lbm_last_error(ctx) -> str:
    return library().lbm_last_error(ctx).decode()


def lbm_destroy(ctx):
    if ctx:
        library().lbm_destroy(ctx)


class Simulation:
    """One context over one or more workload dictionaries."""

    def __init__(self, cfgs, precision="f64", stream=None, phi0=None):
        if isinstance(cfgs, dict):
            cfgs = [cfgs]
        self.cfgs = list(cfgs)
        self.precision = FORMS[precision] if isinstance(precision, str) else int(precision)
        self.ctx = lbm_create([make_params(c) for c in self.cfgs], self.precision, stream)
        if phi0 is not None:
            for k, f in enumerate(phi0):
                lbm_init(self.ctx, k, f)

    def init(self, k, phi0):
        lbm_init(self.ctx, k, phi0)

    def step(self, n):
        lbm_step(self.ctx, n)

    def _shape(self, k):
        c = self.cfgs[k]
        nz = int(c.get("nz", 0))
        return (nz, int(c["ny"]), int(c["nx"])) if nz >= 2 else (int(c["ny"]), int(c["nx"]))

    def fields(self, k=0, names=None) -> dict:
        shape = self._shape(k)
        if names is None:
            names = FIELDS3 if len(shape) == 3 else FIELDS
        mask = 0
        for n in names:
            mask |= FIELD_BITS[n]
        order = [n for n in FIELDS3 if mask & FIELD_BITS[n]]
        out = np.zeros((len(order),) + shape)
        lbm_get_fields(self.ctx, k, mask, out)
        return {n: out[i] for i, n in enumerate(order)}

    def diagnostics(self, k=0) -> dict:
        return lbm_diagnostics(self.ctx, k)

    def populations(self, k=0):
        c = self.cfgs[k]
        return lbm_get_populations(self.ctx, k, int(c["nx"]), int(c["ny"]), int(c.get("nz", 0)))

    def sync(self):
        lbm_sync(self.ctx)

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- single-phase model of Remark 3 (incompressible flow with a mass source) ----
def _check_sp(st, ctx=None):
    if st != LBM_OK:
        msg = library().lbm_sp_last_error(ctx).decode() if ctx else ""
        raise LbmError(st, msg)


class SourceFlow:
    """One single-phase simulation with a mass source on the GPU: Remark 3
    (div u = S; cfg "model": 0), Remark 1 ("model": 1) or Remark 2 ("model": 2,
    "p0"; the source is S_1, the force F_1); cfg "scheme": 1 runs
    Remark 3 with the explicit D_i G_i of Remark 4 and the velocity-dependent
    force F_0 - (drag_lin + drag_quad |u|) u."""

    def __init__(self, cfg: dict, precision="f64", stream=None, source=None):
        p = lbm_sp_params()
        p.nx, p.ny = int(cfg["nx"]), int(cfg["ny"])
        p.bc_y = int(cfg.get("walls_y", 0))
        p.model = int(cfg.get("model", 0))   # 0: Remark 3, 1: Remark 1, 2: Remark 2
        p.p0 = float(cfg.get("p0", 1.0 / 3.0))
        self.model = p.model
        p.nu, p.xi = float(cfg["nu"]), float(cfg.get("xi", 0.0))
        p.force_x, p.force_y = float(cfg.get("force_x", 0.0)), float(cfg.get("force_y", 0.0))
        p.scheme, p.reserved = int(cfg.get("scheme", 0)), 0
        p.drag_lin, p.drag_quad = float(cfg.get("drag_lin", 0.0)), float(cfg.get("drag_quad", 0.0))
        self.nx, self.ny = p.nx, p.ny
        prec = FORMS[precision] if isinstance(precision, str) else int(precision)
        out = _VP()
        st = library().lbm_sp_create(ctypes.byref(p), prec, _VP(stream or 0), ctypes.byref(out))
        if st != LBM_OK:
            raise LbmError(st, "lbm_sp_create")
        self.ctx = out
        if source is not None:
            self.init(source)

    def init(self, source):
        S = np.ascontiguousarray(source, dtype=np.float64)
        assert S.shape == (self.ny, self.nx)
        _check_sp(library().lbm_sp_init(self.ctx, S.ctypes.data_as(_DP)), self.ctx)

    def step(self, n):
        _check_sp(library().lbm_sp_step(self.ctx, int(n)), self.ctx)

    def fields(self) -> dict:
        names = ["ux", "uy", "p"] + (["rho"] if self.model == 1 else [])
        out = np.zeros((len(names), self.ny, self.nx))
        mask = 0
        for n in names:
            mask |= FIELD_BITS[n]
        _check_sp(library().lbm_sp_get_fields(self.ctx, mask, out.ctypes.data_as(_DP)), self.ctx)
        order = [n for n in FIELDS3 if n in names]
        return {n: out[i] for i, n in enumerate(order)}

    def populations(self):
        g = np.zeros((9, self.ny, self.nx))
        _check_sp(library().lbm_sp_get_populations(self.ctx, g.ctypes.data_as(_DP)), self.ctx)
        return g

    def close(self):
        if self.ctx:
            library().lbm_sp_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
