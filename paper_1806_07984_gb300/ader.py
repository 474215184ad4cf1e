"""ctypes binding of the C ABI in include/ader.h (argument marshalling only).

Every function has the name and argument order of its C counterpart and
raises ``AderError`` on a non-zero status.  Pointers are passed as Python
ints (device pointers, e.g. ``tensor.data_ptr()``) or numpy arrays (host
buffers); streams as ``cudaStream_t`` ints (``torch.cuda.Stream.cuda_stream``)
or None for the legacy default stream.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libader.so")

ADER_OK = 0
STATUS_NAMES = {0: "ADER_OK", -1: "ADER_ERR_ARG", -2: "ADER_ERR_CUDA", -3: "ADER_ERR_OOM",
                -4: "ADER_ERR_NONPHYSICAL", -5: "ADER_ERR_PICARD", -6: "ADER_ERR_TIMEOUT",
                -7: "ADER_ERR_MESH"}
ADER_EULER, ADER_ACOUSTICS = 0, 1
ADER_FP64, ADER_FP32, ADER_TF32, ADER_TF32X3, ADER_BF16X3, ADER_DF64 = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp64": ADER_FP64, "fp32": ADER_FP32, "tf32": ADER_TF32, "tf32x3": ADER_TF32X3,
              "bf16x3": ADER_BF16X3, "df64": ADER_DF64}
ADER_ALL, ADER_SKELETON, ADER_ENCLAVE = 0, 1, 2
ADER_PREDICTOR_PICARD, ADER_PREDICTOR_CK = 0, 1
ADER_FIELD_U, ADER_FIELD_USTAR, ADER_FIELD_FACE_Q, ADER_FIELD_FACE_F, ADER_FIELD_FSTAR = range(5)

# Every symbol the header declares (checked by the CPU test suite).
EXPORTS = ["ader_init", "ader_destroy", "ader_error_string", "ader_last_error", "ader_mesh_info",
           "ader_mesh_cells", "ader_mesh_skeleton", "ader_nodes", "ader_set_state",
           "ader_get_state", "ader_get_field", "ader_compute_dt", "ader_predict", "ader_riemann",
           "ader_correct", "ader_step", "ader_step_fixed_dt", "ader_remesh", "ader_classify", "ader_sphere_flags",
           "ader_status_word", "ader_launch_count", "ader_mesh_create", "ader_mesh_destroy",
           "ader_mesh_adapt", "ader_mesh_sizes", "ader_mesh_leaves", "ader_mesh_faces",
           "ader_mesh_sphere_flags", "ader_compute_dt_static", "ader_batch_init",
           "ader_batch_destroy", "ader_batch_last_error", "ader_batch_offsets",
           "ader_batch_set_state", "ader_batch_get_state", "ader_batch_compute_dt",
           "ader_batch_get_dt", "ader_batch_set_launch", "ader_batch_tune", "ader_batch_run",
           "ader_batch_status_word", "ader_batch_launch_count", "ader_adjoint_step",
           "ader_sample", "ader_sample_adjoint", "ader_gradient_flags", "ader_gradient_indicator",
           "ader_limiter_flags",
           "ader_limiter_force", "ader_limiter_refine_flags", "ader_mesh_refine_around",
           "ader_mesh_pipeline", "ader_partition", "ader_dd_info", "ader_dd_cuts",
           "ader_halo_size", "ader_halo_pack", "ader_halo_unpack", "ader_migrate_size",
           "ader_migrate_pack", "ader_migrate_unpack", "ader_mesh_partition",
           "ader_mesh_subdomain", "ader_debug_fail_allocations", "ader_step_refining",
           "ader_step_host"]
ADER_DT_STATIC_MAX_CELLS = 1048576


class AderError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} {detail}".strip())


class ader_batch_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("pde", ctypes.c_int), ("gamma", ctypes.c_double),
                ("picard_iters", ctypes.c_int), ("prec", ctypes.c_int)]


class ader_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("order", ctypes.c_int), ("nvar", ctypes.c_int),
                ("pde", ctypes.c_int), ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
                ("base", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("max_level", ctypes.c_int),
                ("picard_iters", ctypes.c_int), ("prec", ctypes.c_int), ("predictor", ctypes.c_int),
                ("limiter", ctypes.c_int), ("limiter_delta0", ctypes.c_double),
                ("limiter_eps", ctypes.c_double), ("pipeline_chunks", ctypes.c_int),
                ("pipeline_ctas", ctypes.c_int), ("eager_steps", ctypes.c_int)]


_lib = None
_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)


def lib():
    """Load libader.so (once); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1806_07984_gb300.build` (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "ader_init": ([ctypes.POINTER(ader_config), ctypes.POINTER(_vp)], ctypes.c_int),
        "ader_destroy": ([_vp], None),
        "ader_error_string": ([ctypes.c_int], ctypes.c_char_p),
        "ader_last_error": ([_vp], ctypes.c_char_p),
        "ader_mesh_info": ([_vp, _i64p, _i64p, _i64p, _i64p], ctypes.c_int),
        "ader_mesh_cells": ([_vp, _vp], ctypes.c_int),
        "ader_mesh_skeleton": ([_vp, _vp], ctypes.c_int),
        "ader_nodes": ([_vp, _vp], ctypes.c_int),
        "ader_set_state": ([_vp, _vp, ctypes.c_int, _vp], ctypes.c_int),
        "ader_get_state": ([_vp, _vp, ctypes.c_int, _vp], ctypes.c_int),
        "ader_get_field": ([_vp, ctypes.c_int, _vp, ctypes.c_int, _vp], ctypes.c_int),
        "ader_compute_dt": ([_vp, _vp, _vp], ctypes.c_int),
        "ader_predict": ([_vp, _vp, ctypes.c_int, _vp], ctypes.c_int),
        "ader_riemann": ([_vp, ctypes.c_int, _vp], ctypes.c_int),
        "ader_correct": ([_vp, _vp, _vp, _vp], ctypes.c_int),
        "ader_step": ([_vp, ctypes.c_int, _vp, _vp], ctypes.c_int),
        "ader_step_fixed_dt": ([_vp, ctypes.c_int, _vp, _vp, _vp], ctypes.c_int),
        "ader_remesh": ([_vp, _vp], ctypes.c_int),
        "ader_classify": ([_vp, _vp], ctypes.c_int),
        "ader_sphere_flags": ([_vp, _vp, ctypes.c_double, _vp], ctypes.c_int),
        "ader_status_word": ([_vp, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
        "ader_launch_count": ([_vp, _i64p], ctypes.c_int),
        "ader_limiter_flags": ([_vp, _vp, ctypes.c_int, _i64p, _vp], ctypes.c_int),
        "ader_limiter_force": ([_vp, _vp], ctypes.c_int),
        "ader_limiter_refine_flags": ([_vp, _vp], ctypes.c_int),
        "ader_mesh_refine_around": ([_vp, _vp, _vp], ctypes.c_int),
        "ader_mesh_pipeline": ([_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _i64p], ctypes.c_int),
        "ader_mesh_create": ([ctypes.c_int, _vp, ctypes.c_int, ctypes.POINTER(_vp)], ctypes.c_int),
        "ader_mesh_destroy": ([_vp], None),
        "ader_mesh_adapt": ([_vp, _vp], ctypes.c_int),
        "ader_mesh_sizes": ([_vp, _i64p, _i64p, _i64p, _i64p], ctypes.c_int),
        "ader_mesh_leaves": ([_vp, _vp, _vp], ctypes.c_int),
        "ader_mesh_faces": ([_vp, _vp, _vp, _vp], ctypes.c_int),
        "ader_mesh_sphere_flags": ([_vp, _vp, ctypes.c_double, _vp, _vp, _vp], ctypes.c_int),
        "ader_batch_init": ([ctypes.POINTER(ader_batch_config), ctypes.c_int, _vp, _vp, _vp,
                             ctypes.POINTER(_vp)], ctypes.c_int),
        "ader_batch_destroy": ([_vp], None),
        "ader_batch_last_error": ([_vp], ctypes.c_char_p),
        "ader_batch_offsets": ([_vp, _vp], ctypes.c_int),
        "ader_batch_set_state": ([_vp, _vp, ctypes.c_int, _vp], ctypes.c_int),
        "ader_batch_get_state": ([_vp, _vp, ctypes.c_int, _vp], ctypes.c_int),
        "ader_batch_compute_dt": ([_vp, _vp], ctypes.c_int),
        "ader_batch_get_dt": ([_vp, _vp], ctypes.c_int),
        "ader_batch_set_launch": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "ader_batch_tune": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "ader_batch_run": ([_vp, ctypes.c_int, _vp], ctypes.c_int),
        "ader_batch_status_word": ([_vp, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
        "ader_batch_launch_count": ([_vp, _i64p], ctypes.c_int),
        "ader_adjoint_step": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
        "ader_gradient_flags": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 _vp, _vp], ctypes.c_int),
        "ader_gradient_indicator": ([_vp, ctypes.c_int, ctypes.c_int, _vp, _vp], ctypes.c_int),
        "ader_sample": ([_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp, _vp], ctypes.c_int),
        "ader_sample_adjoint": ([_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp, _vp],
                                ctypes.c_int),
        "ader_partition": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "ader_debug_fail_allocations": ([ctypes.c_int], ctypes.c_int),
        "ader_step_host": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
        "ader_step_refining": ([_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _vp], ctypes.c_int),
        "ader_dd_info": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _i64p, _i64p,
                          _i64p, _i64p], ctypes.c_int),
        "ader_dd_cuts": ([_vp, _vp], ctypes.c_int),
        "ader_halo_size": ([_vp, ctypes.c_int, _i64p, _i64p], ctypes.c_int),
        "ader_halo_pack": ([_vp, ctypes.c_int, _vp, _vp], ctypes.c_int),
        "ader_halo_unpack": ([_vp, ctypes.c_int, _vp, _vp], ctypes.c_int),
        "ader_migrate_size": ([_vp, ctypes.c_int, _i64p, _i64p], ctypes.c_int),
        "ader_migrate_pack": ([_vp, ctypes.c_int, _vp, _vp], ctypes.c_int),
        "ader_migrate_unpack": ([_vp, ctypes.c_int, _vp, _vp], ctypes.c_int),
        "ader_mesh_partition": ([_vp, ctypes.c_int, ctypes.c_int, _vp], ctypes.c_int),
        "ader_mesh_subdomain": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
                                ctypes.c_int),
        "ader_compute_dt_static": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp,
                                    _vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _check(ctx, status, where):
    if status != ADER_OK:
        detail = lib().ader_last_error(ctx).decode() if ctx else ""
        raise AderError(status, where, detail)


def ader_init(cfg):
    ctx = _vp()
    _check(None, lib().ader_init(ctypes.byref(cfg), ctypes.byref(ctx)), "ader_init")
    return ctx


def ader_destroy(ctx):
    lib().ader_destroy(ctx)


def ader_error_string(status):
    return lib().ader_error_string(status).decode()


def ader_mesh_info(ctx):
    v = [ctypes.c_int64() for _ in range(4)]
    _check(ctx, lib().ader_mesh_info(ctx, *[ctypes.byref(x) for x in v]), "ader_mesh_info")
    return tuple(x.value for x in v)


def ader_mesh_cells(ctx):
    ncells = ader_mesh_info(ctx)[0]
    out = np.zeros((ncells, 4), dtype=np.int32)
    _check(ctx, lib().ader_mesh_cells(ctx, _ptr(out)), "ader_mesh_cells")
    return out


def ader_mesh_skeleton(ctx):
    ncells = ader_mesh_info(ctx)[0]
    out = np.zeros(ncells, dtype=np.uint8)
    _check(ctx, lib().ader_mesh_skeleton(ctx, _ptr(out)), "ader_mesh_skeleton")
    return out


def ader_nodes(ctx, n):
    out = np.zeros(n, dtype=np.float64)
    _check(ctx, lib().ader_nodes(ctx, _ptr(out)), "ader_nodes")
    return out


def ader_set_state(ctx, u, on_device, stream=None):
    _check(ctx, lib().ader_set_state(ctx, _ptr(u), int(on_device), stream), "ader_set_state")


def ader_get_state(ctx, u, on_device, stream=None):
    _check(ctx, lib().ader_get_state(ctx, _ptr(u), int(on_device), stream), "ader_get_state")


def ader_get_field(ctx, field, out, on_device, stream=None):
    _check(ctx, lib().ader_get_field(ctx, field, _ptr(out), int(on_device), stream),
           "ader_get_field")


def ader_compute_dt(ctx, dt_dev, stream=None):
    _check(ctx, lib().ader_compute_dt(ctx, _ptr(dt_dev), stream), "ader_compute_dt")


def ader_predict(ctx, dt_dev, which=ADER_ALL, stream=None):
    _check(ctx, lib().ader_predict(ctx, _ptr(dt_dev), which, stream), "ader_predict")


def ader_riemann(ctx, which=ADER_ALL, stream=None):
    _check(ctx, lib().ader_riemann(ctx, which, stream), "ader_riemann")


def ader_correct(ctx, dt_dev, dt_next_dev, stream=None):
    _check(ctx, lib().ader_correct(ctx, _ptr(dt_dev), _ptr(dt_next_dev), stream), "ader_correct")


def ader_step(ctx, nsteps, dt_dev, stream=None):
    _check(ctx, lib().ader_step(ctx, nsteps, _ptr(dt_dev), stream), "ader_step")


def ader_step_fixed_dt(ctx, nsteps, dt_dev, dt_next_dev=None, stream=None):
    _check(ctx, lib().ader_step_fixed_dt(ctx, nsteps, _ptr(dt_dev), _ptr(dt_next_dev), stream),
           "ader_step_fixed_dt")


def ader_remesh(ctx, flags):
    flags = np.ascontiguousarray(flags, dtype=np.int8)
    _check(ctx, lib().ader_remesh(ctx, _ptr(flags)), "ader_remesh")


def ader_classify(ctx, flags=None):
    if flags is not None:
        flags = np.ascontiguousarray(flags, dtype=np.int8)
    _check(ctx, lib().ader_classify(ctx, _ptr(flags)), "ader_classify")


def ader_sphere_flags(ctx, center, radius):
    ncells = ader_dd_info(ctx)[2]          # whole mesh (also when partitioned)
    c = np.zeros(3, dtype=np.float64)
    c[:len(center)] = center
    out = np.zeros(ncells, dtype=np.int8)
    _check(ctx, lib().ader_sphere_flags(ctx, _ptr(c), float(radius), _ptr(out)),
           "ader_sphere_flags")
    return out


def ader_status_word(ctx):
    v = ctypes.c_uint32()
    _check(ctx, lib().ader_status_word(ctx, ctypes.byref(v)), "ader_status_word")
    return v.value


def ader_limiter_flags(ctx, stream=None):
    """Per-cell limiter flags of the last corrector (host uint32 array) and the
    number of limited cells."""
    ncells = ader_mesh_info(ctx)[0]
    out = np.zeros(ncells, dtype=np.uint32)
    cnt = ctypes.c_int64()
    _check(ctx, lib().ader_limiter_flags(ctx, _ptr(out), 0, ctypes.byref(cnt), stream),
           "ader_limiter_flags")
    return out, cnt.value


def ader_limiter_force(ctx, force):
    """Cells treated as troubled from now on (bool/uint8 per cell); None clears."""
    if force is None:
        _check(ctx, lib().ader_limiter_force(ctx, None), "ader_limiter_force")
        return
    f = np.ascontiguousarray(np.asarray(force).astype(np.uint8))
    _check(ctx, lib().ader_limiter_force(ctx, _ptr(f)), "ader_limiter_force")


def ader_limiter_refine_flags(ctx):
    """Remesh flags around the cells troubled in the last corrector."""
    out = np.zeros(ader_mesh_info(ctx)[0], dtype=np.int8)
    _check(ctx, lib().ader_limiter_refine_flags(ctx, _ptr(out)), "ader_limiter_refine_flags")
    return out


def ader_launch_count(ctx):
    v = ctypes.c_int64()
    _check(ctx, lib().ader_launch_count(ctx, ctypes.byref(v)), "ader_launch_count")
    return v.value


# ---- host-only mesh handle -------------------------------------------------
def ader_mesh_create(dim, base, max_level):
    b = np.ones(3, dtype=np.int32)
    b[:dim] = base[:dim]
    m = _vp()
    _check(None, lib().ader_mesh_create(dim, _ptr(b), max_level, ctypes.byref(m)),
           "ader_mesh_create")
    return m


def ader_mesh_destroy(mesh):
    lib().ader_mesh_destroy(mesh)


def ader_mesh_adapt(mesh, flags):
    flags = np.ascontiguousarray(flags, dtype=np.int8)
    _check(None, lib().ader_mesh_adapt(mesh, _ptr(flags)), "ader_mesh_adapt")


def ader_mesh_sizes(mesh):
    v = [ctypes.c_int64() for _ in range(4)]
    _check(None, lib().ader_mesh_sizes(mesh, *[ctypes.byref(x) for x in v]), "ader_mesh_sizes")
    return tuple(x.value for x in v)


def ader_mesh_leaves(mesh):
    C = ader_mesh_sizes(mesh)[0]
    cells = np.zeros((C, 4), dtype=np.int32)
    skel = np.zeros(C, dtype=np.uint8)
    _check(None, lib().ader_mesh_leaves(mesh, _ptr(cells), _ptr(skel)), "ader_mesh_leaves")
    return cells, skel


def ader_mesh_faces(mesh, dim):
    C, _, nconf, npar = ader_mesh_sizes(mesh)
    conf = np.zeros((nconf, 3), dtype=np.int32)
    par = np.zeros((npar, 3), dtype=np.int32)
    kids = np.zeros((npar, 3 ** (dim - 1)), dtype=np.int32)
    _check(None, lib().ader_mesh_faces(mesh, _ptr(conf), _ptr(par), _ptr(kids)),
           "ader_mesh_faces")
    return conf, par, kids


def ader_mesh_sphere_flags(mesh, center, radius, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    C = ader_mesh_sizes(mesh)[0]
    c = np.zeros(3)
    c[:len(center)] = center
    lo_ = np.zeros(3)
    lo_[:len(lo)] = lo
    hi_ = np.ones(3)
    hi_[:len(hi)] = hi
    out = np.zeros(C, dtype=np.int8)
    _check(None, lib().ader_mesh_sphere_flags(mesh, _ptr(c), float(radius), _ptr(lo_), _ptr(hi_),
                                              _ptr(out)), "ader_mesh_sphere_flags")
    return out


def ader_compute_dt_static(dim, order, pde, gamma, cfl, base, lo, hi, ncells, u_dev, level_dev,
                           dt_dev, stream=None):
    """Allocation-free global time step (no context); see include/ader.h."""
    b = np.ones(3, dtype=np.int32)
    b[:dim] = base[:dim]
    lo_ = np.zeros(3)
    lo_[:dim] = lo[:dim]
    hi_ = np.ones(3)
    hi_[:dim] = hi[:dim]
    _check(None, lib().ader_compute_dt_static(dim, order, pde, gamma, cfl, _ptr(b), _ptr(lo_),
                                              _ptr(hi_), ncells, _ptr(u_dev), _ptr(level_dev),
                                              _ptr(dt_dev), stream), "ader_compute_dt_static")


# ---- batched instances ------------------------------------------------------
def _bcheck(b, status, where):
    if status != ADER_OK:
        detail = lib().ader_batch_last_error(b).decode() if b else ""
        raise AderError(status, where, detail)


def ader_batch_init(cfg, sides, orders, cfls):
    sides = np.ascontiguousarray(sides, dtype=np.int32)
    orders = np.ascontiguousarray(orders, dtype=np.int32)
    cfls = np.ascontiguousarray(cfls, dtype=np.float64)
    b = _vp()
    _bcheck(None, lib().ader_batch_init(ctypes.byref(cfg), len(sides), _ptr(sides), _ptr(orders),
                                        _ptr(cfls), ctypes.byref(b)), "ader_batch_init")
    return b


def ader_batch_destroy(b):
    lib().ader_batch_destroy(b)


def ader_batch_offsets(b, ninst):
    out = np.zeros(ninst + 1, dtype=np.int64)
    _bcheck(b, lib().ader_batch_offsets(b, _ptr(out)), "ader_batch_offsets")
    return out


def ader_batch_set_state(b, u, on_device, stream=None):
    _bcheck(b, lib().ader_batch_set_state(b, _ptr(u), int(on_device), stream), "ader_batch_set_state")


def ader_batch_get_state(b, u, on_device, stream=None):
    _bcheck(b, lib().ader_batch_get_state(b, _ptr(u), int(on_device), stream), "ader_batch_get_state")


def ader_batch_compute_dt(b, stream=None):
    _bcheck(b, lib().ader_batch_compute_dt(b, stream), "ader_batch_compute_dt")


def ader_batch_get_dt(b, ninst):
    out = np.zeros(ninst, dtype=np.float64)
    _bcheck(b, lib().ader_batch_get_dt(b, _ptr(out)), "ader_batch_get_dt")
    return out


def ader_batch_set_launch(b, blocks_per_sm, tile):
    _bcheck(b, lib().ader_batch_set_launch(b, blocks_per_sm, tile), "ader_batch_set_launch")


def ader_batch_tune(b):
    bps, tile, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _bcheck(b, lib().ader_batch_tune(b, ctypes.byref(bps), ctypes.byref(tile), ctypes.byref(ms)),
            "ader_batch_tune")
    return bps.value, tile.value, ms.value


def ader_batch_run(b, nsteps, stream=None):
    _bcheck(b, lib().ader_batch_run(b, nsteps, stream), "ader_batch_run")


def ader_batch_status_word(b):
    v = ctypes.c_uint32()
    _bcheck(b, lib().ader_batch_status_word(b, ctypes.byref(v)), "ader_batch_status_word")
    return v.value


def ader_batch_launch_count(b):
    v = ctypes.c_int64()
    _bcheck(b, lib().ader_batch_launch_count(b, ctypes.byref(v)), "ader_batch_launch_count")
    return v.value


# ---- adjoint and point sampling --------------------------------------------
def ader_adjoint_step(ctx, lam_in, lam_out, dt_dev, stream=None):
    _check(ctx, lib().ader_adjoint_step(ctx, _ptr(lam_in), _ptr(lam_out), _ptr(dt_dev), stream),
           "ader_adjoint_step")


def ader_sample(ctx, npts, cells_dev, weights_dev, var, field_dev, out_dev, stream=None):
    _check(ctx, lib().ader_sample(ctx, npts, _ptr(cells_dev), _ptr(weights_dev), var,
                                  _ptr(field_dev), _ptr(out_dev), stream), "ader_sample")


def ader_sample_adjoint(ctx, npts, cells_dev, weights_dev, var, values_dev, field_dev, stream=None):
    _check(ctx, lib().ader_sample_adjoint(ctx, npts, _ptr(cells_dev), _ptr(weights_dev), var,
                                          _ptr(values_dev), _ptr(field_dev), stream),
           "ader_sample_adjoint")


def ader_gradient_flags(ctx, var, refine_above, coarsen_below, deriv=1):
    ncells = ader_mesh_info(ctx)[0]
    eta = np.zeros(ncells, dtype=np.float64)
    flags = np.zeros(ncells, dtype=np.int8)
    _check(ctx, lib().ader_gradient_flags(ctx, var, int(deriv), float(refine_above),
                                          float(coarsen_below), _ptr(eta), _ptr(flags)),
           "ader_gradient_flags")
    return eta, flags


def ader_gradient_indicator(ctx, var, eta_dev, stream=None, deriv=1):
    """eta (device array of ncells doubles) of ader_gradient_flags, enqueued on
    ``stream`` (a raw cudaStream_t handle; None = legacy default stream)."""
    _check(ctx, lib().ader_gradient_indicator(ctx, var, int(deriv), _ptr(eta_dev), stream),
           "ader_gradient_indicator")


def ader_mesh_refine_around(mesh, troubled):
    t = np.ascontiguousarray(np.asarray(troubled).astype(np.uint8))
    out = np.zeros(len(t), dtype=np.int8)
    _check(None, lib().ader_mesh_refine_around(mesh, _ptr(t), _ptr(out)), "ader_mesh_refine_around")
    return out


def ader_mesh_pipeline(mesh, K):
    """(chunk_off, face_off, corr_off, corr_cells, conf, n_skeleton_faces) of
    the enclave pipeline with K chunks."""
    C, _, nconf, _ = ader_mesh_sizes(mesh)
    chunk = np.zeros(K + 1, dtype=np.int64)
    face = np.zeros(K + 1, dtype=np.int64)
    corr = np.zeros(K + 2, dtype=np.int64)
    cells = np.zeros(C, dtype=np.int32)
    conf = np.zeros((nconf, 3), dtype=np.int32)
    nsk = ctypes.c_int64()
    _check(None, lib().ader_mesh_pipeline(mesh, K, _ptr(chunk), _ptr(face), _ptr(corr), _ptr(cells),
                                          _ptr(conf), ctypes.byref(nsk)), "ader_mesh_pipeline")
    return chunk, face, corr, cells, conf, nsk.value


# ---- domain decomposition ---------------------------------------------------
def ader_partition(ctx, nranks, rank):
    _check(ctx, lib().ader_partition(ctx, nranks, rank), "ader_partition")


def ader_dd_info(ctx):
    """(nranks, rank, nglobal, first, nowned, nghost)."""
    r = [ctypes.c_int(), ctypes.c_int()]
    v = [ctypes.c_int64() for _ in range(4)]
    _check(ctx, lib().ader_dd_info(ctx, *[ctypes.byref(x) for x in r + v]), "ader_dd_info")
    return tuple(x.value for x in r + v)


def ader_dd_cuts(ctx):
    cuts = np.zeros(ader_dd_info(ctx)[0] + 1, dtype=np.int64)
    _check(ctx, lib().ader_dd_cuts(ctx, _ptr(cuts)), "ader_dd_cuts")
    return cuts


def ader_halo_size(ctx, peer):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, lib().ader_halo_size(ctx, peer, ctypes.byref(a), ctypes.byref(b)), "ader_halo_size")
    return a.value, b.value


def ader_halo_pack(ctx, peer, buf, stream=None):
    _check(ctx, lib().ader_halo_pack(ctx, peer, _ptr(buf), stream), "ader_halo_pack")


def ader_halo_unpack(ctx, peer, buf, stream=None):
    _check(ctx, lib().ader_halo_unpack(ctx, peer, _ptr(buf), stream), "ader_halo_unpack")


def ader_migrate_size(ctx, peer):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, lib().ader_migrate_size(ctx, peer, ctypes.byref(a), ctypes.byref(b)),
           "ader_migrate_size")
    return a.value, b.value


def ader_migrate_pack(ctx, peer, buf, stream=None):
    _check(ctx, lib().ader_migrate_pack(ctx, peer, _ptr(buf), stream), "ader_migrate_pack")


def ader_migrate_unpack(ctx, peer, buf, stream=None):
    _check(ctx, lib().ader_migrate_unpack(ctx, peer, _ptr(buf), stream), "ader_migrate_unpack")


def ader_mesh_partition(mesh, nranks, rank, dim):
    """Host partition of a mesh handle: a dict of the sub-domain lists (see
    include/ader.h) for rank ``rank`` of ``nranks``."""
    sz = np.zeros(9, dtype=np.int64)
    _check(None, lib().ader_mesh_partition(mesh, nranks, rank, _ptr(sz)), "ader_mesh_partition")
    first, nown, nghost, nconf, nconf_skel, npar, nskel, nsend, nrecv = (int(x) for x in sz)
    out = dict(first=first, nowned=nown, nghost=nghost, n_conf_skeleton=nconf_skel,
               cuts=np.zeros(nranks + 1, dtype=np.int64), ghosts=np.zeros(nghost, dtype=np.int32),
               conf=np.zeros((nconf, 3), dtype=np.int32), parents=np.zeros((npar, 3), dtype=np.int32),
               children=np.zeros((npar, 3 ** (dim - 1)), dtype=np.int32),
               skeleton=np.zeros(nskel, dtype=np.int32),
               send_off=np.zeros(nranks + 1, dtype=np.int64), send=np.zeros(nsend, dtype=np.int32),
               recv_off=np.zeros(nranks + 1, dtype=np.int64), recv=np.zeros(nrecv, dtype=np.int32))
    _check(None, lib().ader_mesh_subdomain(
        mesh, _ptr(out["cuts"]), _ptr(out["ghosts"]), _ptr(out["conf"]), _ptr(out["parents"]),
        _ptr(out["children"]), _ptr(out["skeleton"]), _ptr(out["send_off"]), _ptr(out["send"]),
        _ptr(out["recv_off"]), _ptr(out["recv"])), "ader_mesh_subdomain")
    return out


def ader_debug_fail_allocations(after):
    """Fault injection for tests: the library's device allocations fail after
    `after` more successes (after < 0: off)."""
    _check(None, lib().ader_debug_fail_allocations(after), "ader_debug_fail_allocations")


def ader_step_refining(ctx, dt, max_rounds, stream=None):
    """One limited step with immediate refinement around troubled cells at
    resolution transitions; returns the number of refinements."""
    r = ctypes.c_int()
    _check(ctx, lib().ader_step_refining(ctx, _ptr(dt), max_rounds, ctypes.byref(r), stream),
           "ader_step_refining")
    return r.value


def ader_step_host(ctx, u_in, u_out, dt, stream=None):
    """One step with the state read from u_in and written to u_out (host
    buffers, page-locked for the copies to overlap the predictor)."""
    _check(ctx, lib().ader_step_host(ctx, _ptr(u_in), _ptr(u_out), _ptr(dt), stream), "ader_step_host")
