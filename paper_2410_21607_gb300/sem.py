"""ctypes binding of libsem.so (include/sem.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: device arrays are torch CUDA tensors (float64,
contiguous, shape (5, NG) for fields), streams are torch CUDA streams (the
current stream by default).  If the shared library is missing this module
raises on import: there is no fallback path.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libsem.so")

SEM_OK, SEM_ERR_ARG, SEM_ERR_CUDA, SEM_ERR_TOPOLOGY = 0, 1, 2, 3
SEM_ERR_NUMERIC, SEM_ERR_TIMEOUT, SEM_ERR_IO, SEM_ERR_UNSUPPORTED = 4, 5, 6, 7
SEM_EQ_CONSERVATIVE, SEM_EQ_NONCONSERVATIVE = 0, 1
SEM_PREC_FP64, SEM_PREC_MIXED = 0, 1
SEM_MAX_THRESHOLDS = 8
SEM_CRIT_SPEED, SEM_CRIT_VORTICITY, SEM_CRIT_PV = 0, 1, 2

# every symbol include/sem.h declares
EXPORTS = (
    "sem_last_error", "sem_params_default", "sem_mesh_create", "sem_mesh_destroy",
    "sem_mesh_get_info", "sem_mesh_coords_host", "sem_mesh_leaves_host", "sem_mesh_hmap_host",
    "sem_mesh_mass_host", "sem_mesh_coords", "sem_rhs", "sem_rhs_noalloc", "sem_rk_stage",
    "sem_rk_stage_mixed",
    "sem_mirror", "sem_step", "sem_step_mixed",
    "sem_adapt_flags", "sem_adapt_flags_host", "sem_transfer_plan", "sem_transfer", "sem_diag",
    "sem_status", "sem_profile_begin", "sem_profile_end", "sem_autotune", "sem_autotune_select",
    "sem_batch_create", "sem_batch_destroy", "sem_batch_step_mixed", "sem_batch_status",
    "sem_mlp_create", "sem_mlp_destroy", "sem_mlp_param_count", "sem_mlp_get_params",
    "sem_mlp_set_params", "sem_mlp_get_grads", "sem_mlp_features", "sem_mlp_forward",
    "sem_mlp_predict_flags", "sem_mlp_backward", "sem_mlp_adam",
    "sem_checkpoint_write", "sem_checkpoint_read_mesh", "sem_checkpoint_read_state",
    "sem_selftest_device_once", "sem_peak_probe", "sem_adapt_flags_levels", "sem_merge_flags",
    "sem_mlp_select_forward", "sem_mlp_status",
)


class SemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sem error {code}: {msg}")
        self.code = code


class MeshDesc(C.Structure):
    _fields_ = [("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("N", C.c_int),
                ("periodic_x", C.c_int), ("periodic_y", C.c_int), ("lvl_max", C.c_int),
                ("n_leaves", C.c_int), ("leaves", C.POINTER(C.c_int)),
                ("z_faces", C.POINTER(C.c_double)),
                ("warp_amplitude", C.c_double), ("warp_kx", C.c_int), ("warp_ky", C.c_int)]


class MeshInfo(C.Structure):
    _fields_ = [("Ne", C.c_longlong), ("NL", C.c_longlong), ("NG", C.c_longlong),
                ("NH", C.c_longlong), ("NZ", C.c_longlong), ("Ncol", C.c_longlong),
                ("n_hanging_h", C.c_longlong), ("n_nonconforming_faces", C.c_longlong),
                ("N", C.c_int), ("nz", C.c_int), ("max_level", C.c_int),
                ("level_hist", C.c_longlong * 16)]


class Params(C.Structure):
    _fields_ = [("g", C.c_double), ("f", C.c_double), ("R_d", C.c_double), ("c_p", C.c_double),
                ("p00", C.c_double), ("theta_s", C.c_double), ("N_bv", C.c_double),
                ("eqset", C.c_int), ("precision", C.c_int), ("n_thresholds", C.c_int),
                ("lvl_max", C.c_int), ("thresholds", C.c_double * SEM_MAX_THRESHOLDS),
                ("smag_cs", C.c_double), ("sponge_gamma", C.c_double), ("sponge_depth", C.c_double),
                ("criterion", C.c_int * SEM_MAX_THRESHOLDS),
                ("heat_q0", C.c_double), ("heat_r0", C.c_double), ("heat_width", C.c_double),
                ("heat_rmax", C.c_double), ("heat_ztop", C.c_double), ("heat_ramp", C.c_double),
                ("time", C.c_double)]


class ProfileOut(C.Structure):
    _fields_ = [("n_kernels", C.c_int), ("name", (C.c_char * 48) * 16),
                ("launches", C.c_longlong * 16), ("ms_total", C.c_double * 16)]


class TuneOut(C.Structure):
    _fields_ = [("n_variants", C.c_int), ("chosen", C.c_int), ("layers_per_cta", C.c_int * 16),
                ("min_ctas_per_sm", C.c_int * 16), ("kind", C.c_int * 16),
                ("ms", C.c_double * 16)]


class DiagOut(C.Structure):
    _fields_ = [("max_wind", C.c_double), ("max_mean_wind", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2410_21607_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    sig = {
        "sem_last_error": (C.c_char_p, []),
        "sem_params_default": (i, [C.POINTER(Params)]),
        "sem_mesh_create": (i, [C.POINTER(MeshDesc), C.POINTER(vp)]),
        "sem_mesh_destroy": (None, [vp]),
        "sem_mesh_get_info": (i, [vp, C.POINTER(MeshInfo)]),
        "sem_mesh_coords_host": (i, [vp, vp]),
        "sem_mesh_leaves_host": (i, [vp, vp]),
        "sem_mesh_hmap_host": (i, [vp, vp, vp, vp]),
        "sem_mesh_mass_host": (i, [vp, vp]),
        "sem_mesh_coords": (i, [vp, vp, vp]),
        "sem_rhs": (i, [vp, C.POINTER(Params), vp, vp, vp]),
        "sem_rhs_noalloc": (i, [vp, C.POINTER(Params), vp, vp, vp]),
        "sem_rk_stage": (i, [vp, C.POINTER(Params), i, vp, vp, vp, d, vp]),
        "sem_rk_stage_mixed": (i, [vp, C.POINTER(Params), i, vp, vp, vp, vp, vp, d, vp]),
        "sem_mirror": (i, [vp, vp, vp, vp]),
        "sem_step_mixed": (i, [vp, C.POINTER(Params), vp, vp, vp, d, vp]),
        "sem_step": (i, [vp, C.POINTER(Params), vp, vp, vp, d, vp]),
        "sem_adapt_flags": (i, [vp, C.POINTER(Params), vp, vp, vp, vp]),
        "sem_adapt_flags_host": (i, [vp, C.POINTER(Params), vp, vp, vp]),
        "sem_transfer_plan": (i, [vp, vp, C.POINTER(vp)]),
        "sem_transfer": (i, [vp, vp, vp, vp, vp]),
        "sem_diag": (i, [vp, C.POINTER(Params), vp, d, C.POINTER(DiagOut), vp]),
        "sem_status": (i, [vp, C.POINTER(C.c_int), vp]),
        "sem_profile_begin": (i, []),
        "sem_batch_create": (i, [C.POINTER(vp), i, C.POINTER(vp)]),
        "sem_batch_destroy": (None, [vp]),
        "sem_batch_step_mixed": (i, [vp, C.POINTER(Params), C.POINTER(vp), C.POINTER(vp),
                                     C.POINTER(vp), C.POINTER(d), i, vp]),
        "sem_batch_status": (i, [vp, C.POINTER(C.c_int), vp]),
        "sem_mlp_create": (i, [C.c_ulonglong, i, C.POINTER(vp)]),
        "sem_mlp_destroy": (None, [vp]),
        "sem_mlp_param_count": (i, []),
        "sem_mlp_get_params": (i, [vp, vp]),
        "sem_mlp_set_params": (i, [vp, vp]),
        "sem_mlp_get_grads": (i, [vp, vp]),
        "sem_mlp_features": (i, [vp, vp, vp, vp, vp]),
        "sem_mlp_forward": (i, [vp, vp, i, vp, vp]),
        "sem_mlp_predict_flags": (i, [vp, vp, i, vp, vp]),
        "sem_mlp_backward": (i, [vp, vp, vp, vp, i, C.POINTER(d), vp]),
        "sem_mlp_adam": (i, [vp, C.c_float, vp]),
        "sem_checkpoint_write": (i, [vp, vp, d, C.c_longlong, C.c_char_p, vp]),
        "sem_checkpoint_read_mesh": (i, [C.c_char_p, C.POINTER(vp), C.POINTER(d), C.POINTER(C.c_longlong)]),
        "sem_checkpoint_read_state": (i, [C.c_char_p, vp, vp, vp]),
        "sem_autotune": (i, [vp, C.POINTER(Params), vp, i, C.POINTER(TuneOut), vp]),
        "sem_autotune_select": (i, [vp, i, i]),
        "sem_selftest_device_once": (i, [i, i, vp]),
        "sem_peak_probe": (i, [i, C.POINTER(d), vp]),
        "sem_adapt_flags_levels": (i, [vp, C.POINTER(Params), vp, vp, i, vp, vp, vp]),
        "sem_merge_flags": (i, [vp, vp, vp, i, C.c_longlong, vp, vp]),
        "sem_mlp_select_forward": (i, [vp, i]),
        "sem_mlp_status": (i, [vp, C.POINTER(C.c_int), vp]),
        "sem_profile_end": (i, [C.POINTER(ProfileOut)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


def _check(rc):
    if rc != SEM_OK:
        raise SemError(rc, LIB.sem_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("host array must be C-contiguous")
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _torch():
    import torch
    return torch


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _f64(t, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError("expected a float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
    return t


def sem_params_default(**overrides):
    p = Params()
    _check(LIB.sem_params_default(C.byref(p)))
    thr = overrides.pop("thresholds", None)
    crit = overrides.pop("criterion", None)
    for k, v in overrides.items():
        setattr(p, k, v)
    if crit is not None:
        for k, v in enumerate(crit):
            p.criterion[k] = v
    if thr is not None:
        p.n_thresholds = len(thr)
        for k, v in enumerate(thr):
            p.thresholds[k] = v
    return p


class Mesh:
    """Owning handle of a sem_mesh."""

    def __init__(self, handle):
        self.h = C.c_void_p(handle)
        info = MeshInfo()
        _check(LIB.sem_mesh_get_info(self.h, C.byref(info)))
        self.info = info
        self.NG, self.NH, self.NZ, self.Ne = info.NG, info.NH, info.NZ, info.Ne
        self.N, self.nz, self.Ncol = info.N, info.nz, info.Ncol

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            LIB.sem_mesh_destroy(h)
            self.h = None

    @property
    def field_shape(self):
        return (5, self.NG)


def sem_mesh_create(Lx, Ly, Lz, nx, ny, nz, N, leaves=None, periodic=(True, True), lvl_max=0,
                    z_faces=None, warp=None):
    """warp = (amplitude, kx, ky): warped layers (sem_mesh_desc), None: boxes."""
    wa, wx, wy = (0.0, 1, 1) if warp is None else (float(warp[0]), int(warp[1]), int(warp[2]))
    d = MeshDesc(Lx, Ly, Lz, nx, ny, nz, N, int(periodic[0]), int(periodic[1]), lvl_max, 0, None, None,
                 wa, wx, wy)
    keep = keep_z = None
    if leaves is not None and len(leaves):
        keep = np.ascontiguousarray(np.asarray(leaves, dtype=np.int32).reshape(-1, 3))
        d.n_leaves = len(keep)
        d.leaves = keep.ctypes.data_as(C.POINTER(C.c_int))
    if z_faces is not None:
        keep_z = np.ascontiguousarray(np.asarray(z_faces, dtype=np.float64))
        if keep_z.shape != (nz + 1,):
            raise ValueError("z_faces needs nz + 1 values")
        d.z_faces = keep_z.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()
    _check(LIB.sem_mesh_create(C.byref(d), C.byref(h)))
    return Mesh(h.value)


def sem_mesh_coords_host(mesh):
    out = np.zeros((3, mesh.NG))
    _check(LIB.sem_mesh_coords_host(mesh.h, _ptr(out)))
    return out


def sem_mesh_leaves_host(mesh):
    out = np.zeros((mesh.Ncol, 3), dtype=np.int32)
    _check(LIB.sem_mesh_leaves_host(mesh.h, _ptr(out)))
    return out


def sem_mesh_hmap_host(mesh):
    n1 = mesh.N + 1
    hmap = np.zeros((mesh.Ncol, n1 * n1), dtype=np.int32)
    nh = mesh.info.n_hanging_h
    hh = np.zeros((max(nh, 1), n1), dtype=np.int32)
    hw = np.zeros((max(nh, 1), n1))
    _check(LIB.sem_mesh_hmap_host(mesh.h, _ptr(hmap), _ptr(hh), _ptr(hw)))
    return hmap, hh[:nh], hw[:nh]


def sem_mesh_mass_host(mesh):
    out = np.zeros(mesh.NG)
    _check(LIB.sem_mesh_mass_host(mesh.h, _ptr(out)))
    return out


def sem_mesh_coords(mesh, out, stream=None):
    _f64(out, (3, mesh.NG))
    _check(LIB.sem_mesh_coords(mesh.h, _ptr(out), _stream(stream)))
    return out


def sem_rhs(mesh, params, q, out, stream=None):
    _f64(q, mesh.field_shape)
    _f64(out, mesh.field_shape)
    _check(LIB.sem_rhs(mesh.h, C.byref(params), _ptr(q), _ptr(out), _stream(stream)))
    return out


def sem_rhs_noalloc(mesh, params, q, out, stream=None):
    """sem_rhs with the library's fixed 16 MiB device scratch instead of the
    mesh's own: for callers that may not allocate device memory at this point.
    The mesh needs its device tables already (any earlier device call)."""
    _f64(q, mesh.field_shape)
    _f64(out, mesh.field_shape)
    _check(LIB.sem_rhs_noalloc(mesh.h, C.byref(params), _ptr(q), _ptr(out), _stream(stream)))
    return out


def sem_rk_stage(mesh, params, stage, qn, qs, qout, dt, stream=None):
    for t in (qn, qs, qout):
        _f64(t, mesh.field_shape)
    _check(LIB.sem_rk_stage(mesh.h, C.byref(params), int(stage), _ptr(qn), _ptr(qs), _ptr(qout),
                            float(dt), _stream(stream)))
    return qout


def _f32(t, shape):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda:
        raise TypeError("expected a float32 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
    return t


def sem_rk_stage_mixed(mesh, params, stage, qn, qs, qs32, qout, qout32, dt, stream=None):
    for t in (qn, qs, qout):
        _f64(t, mesh.field_shape)
    for t in (qs32, qout32):
        _f32(t, mesh.field_shape)
    _check(LIB.sem_rk_stage_mixed(mesh.h, C.byref(params), int(stage), _ptr(qn), _ptr(qs),
                                  _ptr(qs32), _ptr(qout), _ptr(qout32), float(dt), _stream(stream)))
    return qout


def sem_step_mixed(mesh, params, q, q32, work32, dt, stream=None):
    _f64(q, mesh.field_shape)
    _f32(q32, mesh.field_shape)
    _f32(work32, (2 * 5, mesh.NG))
    _check(LIB.sem_step_mixed(mesh.h, C.byref(params), _ptr(q), _ptr(q32), _ptr(work32),
                              float(dt), _stream(stream)))
    return q


def sem_mirror(mesh, q, q32, stream=None):
    _f64(q, mesh.field_shape)
    _f32(q32, mesh.field_shape)
    _check(LIB.sem_mirror(mesh.h, _ptr(q), _ptr(q32), _stream(stream)))
    return q32


def sem_step(mesh, params, q, w1, w2, dt, stream=None):
    for t in (q, w1, w2):
        _f64(t, mesh.field_shape)
    _check(LIB.sem_step(mesh.h, C.byref(params), _ptr(q), _ptr(w1), _ptr(w2), float(dt),
                        _stream(stream)))
    return q


def sem_adapt_flags(mesh, params, q, flags, cmax=None, stream=None):
    _f64(q, mesh.field_shape)
    _check(LIB.sem_adapt_flags(mesh.h, C.byref(params), _ptr(q), _ptr(flags), _ptr(cmax),
                               _stream(stream)))
    return flags


def sem_adapt_flags_levels(mesh, params, q, flags, level=None, level_all=-1, cmax=None, stream=None):
    """The criterion's flags for the per-element levels `level` (int8 device
    tensor [Ne]) or, with level None, for every element at level_all."""
    _f64(q, mesh.field_shape)
    if level is not None and (level.dtype != _torch().int8 or level.numel() != mesh.Ne):
        raise ValueError("level: int8 tensor of one level per element")
    _check(LIB.sem_adapt_flags_levels(mesh.h, C.byref(params), _ptr(q), _ptr(level), int(level_all),
                                      _ptr(flags), _ptr(cmax), _stream(stream)))
    return flags


def sem_merge_flags(crit, pred, level, lvl_max, out=None, stream=None):
    """Criterion flags merged with a predictor's (int8 device tensors [n]):
    refine if either asks, coarsen only if both do, within the level bounds."""
    n = crit.numel()
    for t in (crit, pred, level):
        if t.dtype != _torch().int8 or t.numel() != n:
            raise ValueError("crit, pred and level: int8 tensors of equal length")
    if out is None:
        out = _torch().empty_like(crit)
    _check(LIB.sem_merge_flags(_ptr(crit), _ptr(pred), _ptr(level), int(lvl_max), n, _ptr(out),
                               _stream(stream)))
    return out


def sem_adapt_flags_host(mesh, params, q, stream=None):
    _f64(q, mesh.field_shape)
    out = np.zeros(mesh.Ne, dtype=np.int8)
    _check(LIB.sem_adapt_flags_host(mesh.h, C.byref(params), _ptr(q), _ptr(out), _stream(stream)))
    return out


def sem_transfer_plan(mesh, flags_host):
    f = np.ascontiguousarray(np.asarray(flags_host, dtype=np.int8))
    if f.shape != (mesh.Ne,):
        raise ValueError("one flag per element")
    h = C.c_void_p()
    _check(LIB.sem_transfer_plan(mesh.h, _ptr(f), C.byref(h)))
    return Mesh(h.value)


def sem_transfer(old, new, q_old, q_new, stream=None):
    _f64(q_old, old.field_shape)
    _f64(q_new, new.field_shape)
    _check(LIB.sem_transfer(old.h, new.h, _ptr(q_old), _ptr(q_new), _stream(stream)))
    return q_new


def sem_diag(mesh, params, q, half_width=50.0e3, stream=None):
    _f64(q, mesh.field_shape)
    out = DiagOut()
    _check(LIB.sem_diag(mesh.h, C.byref(params), _ptr(q), float(half_width), C.byref(out),
                        _stream(stream)))
    return {"max_wind": out.max_wind, "max_mean_wind": out.max_mean_wind}


def sem_status(mesh, stream=None):
    v = C.c_int(0)
    _check(LIB.sem_status(mesh.h, C.byref(v), _stream(stream)))
    return v.value


def sem_profile_begin():
    _check(LIB.sem_profile_begin())


def sem_profile_end():
    """{kernel name: (launches, total ms)} of the launches since sem_profile_begin."""
    out = ProfileOut()
    _check(LIB.sem_profile_end(C.byref(out)))
    return {bytes(out.name[k]).split(b"\0")[0].decode(): (out.launches[k], out.ms_total[k])
            for k in range(out.n_kernels)}


def sem_autotune(mesh, params, q32, reps=5, stream=None):
    """Time the element-kernel variants on this mesh and keep the fastest.
    Returns [(layers_per_cta, min_ctas_per_sm, ms, kind)] and the chosen index
    (kind 0: z-pencil kernel, 1: line-exchange kernel, 2: line exchange with
    the x, y contractions on tensor cores, 4: line exchange with the state
    staged by bulk copies, 5: line exchange for the paper's equation set).
    The table is the one of params.eqset's equation set."""
    _f32(q32, mesh.field_shape)
    out = TuneOut()
    _check(LIB.sem_autotune(mesh.h, C.byref(params), _ptr(q32), int(reps), C.byref(out),
                            _stream(stream)))
    rows = [(out.layers_per_cta[k], out.min_ctas_per_sm[k], out.ms[k], out.kind[k])
            for k in range(out.n_variants)]
    return rows, out.chosen


def sem_autotune_select(mesh, row, eqset=0):
    """Use row `row` of sem_autotune's table for equation set `eqset`
    (0: conservative, 1: the paper's set; row -1: the untuned default)."""
    _check(LIB.sem_autotune_select(mesh.h, int(eqset), int(row)))


class Batch:
    """Owning handle of a sem_batch; keeps its meshes alive."""

    def __init__(self, handle, meshes):
        self.h = C.c_void_p(handle)
        self.meshes = list(meshes)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            LIB.sem_batch_destroy(h)
            self.h = None


def sem_batch_create(meshes):
    arr = (C.c_void_p * len(meshes))(*[m.h.value for m in meshes])
    h = C.c_void_p()
    _check(LIB.sem_batch_create(arr, len(meshes), C.byref(h)))
    return Batch(h.value, meshes)


def sem_batch_step_mixed(batch, params, qs, q32s, works, dts, use_graph=True, stream=None):
    n = len(batch.meshes)
    if not (len(qs) == len(q32s) == len(works) == len(dts) == n):
        raise ValueError("one array set and dt per instance")
    for m, q, q32, w in zip(batch.meshes, qs, q32s, works):
        _f64(q, m.field_shape)
        _f32(q32, m.field_shape)
        _f32(w, (10, m.NG))
    aq = (C.c_void_p * n)(*[q.data_ptr() for q in qs])
    a32 = (C.c_void_p * n)(*[q.data_ptr() for q in q32s])
    aw = (C.c_void_p * n)(*[w.data_ptr() for w in works])
    adt = (C.c_double * n)(*[float(x) for x in dts])
    _check(LIB.sem_batch_step_mixed(batch.h, C.byref(params), aq, a32, aw, adt, int(bool(use_graph)),
                                    _stream(stream)))


def sem_batch_status(batch, stream=None):
    v = C.c_int(0)
    _check(LIB.sem_batch_status(batch.h, C.byref(v), _stream(stream)))
    return v.value


class Mlp:
    """Owning handle of a sem_mlp."""

    def __init__(self, handle, max_rows):
        self.h = C.c_void_p(handle)
        self.max_rows = max_rows
        self.nparam = LIB.sem_mlp_param_count()

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            LIB.sem_mlp_destroy(h)
            self.h = None


def sem_mlp_create(seed, max_rows):
    h = C.c_void_p()
    _check(LIB.sem_mlp_create(int(seed), int(max_rows), C.byref(h)))
    return Mlp(h.value, max_rows)


def sem_mlp_get_params(mlp):
    out = np.zeros(mlp.nparam, dtype=np.float32)
    _check(LIB.sem_mlp_get_params(mlp.h, _ptr(out)))
    return out


def sem_mlp_set_params(mlp, params):
    a = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    if a.size != mlp.nparam:
        raise ValueError("wrong parameter count")
    _check(LIB.sem_mlp_set_params(mlp.h, _ptr(a)))


def sem_mlp_get_grads(mlp):
    out = np.zeros(mlp.nparam, dtype=np.float32)
    _check(LIB.sem_mlp_get_grads(mlp.h, _ptr(out)))
    return out


def sem_mlp_features(mesh, q, scales, feats, stream=None):
    _f64(q, mesh.field_shape)
    _f32(feats, (mesh.Ne, 136))
    sc = np.ascontiguousarray(np.asarray(scales, dtype=np.float32))
    _check(LIB.sem_mlp_features(mesh.h, _ptr(q), _ptr(sc), _ptr(feats), _stream(stream)))
    return feats


def sem_mlp_forward(mlp, feats, prob, stream=None):
    n = feats.shape[0]
    _f32(feats, (n, 136))
    _f32(prob, (n, 3))
    _check(LIB.sem_mlp_forward(mlp.h, _ptr(feats), n, _ptr(prob), _stream(stream)))
    return prob


def sem_mlp_predict_flags(mlp, feats, flags, stream=None):
    n = feats.shape[0]
    _f32(feats, (n, 136))
    _check(LIB.sem_mlp_predict_flags(mlp.h, _ptr(feats), n, _ptr(flags), _stream(stream)))
    return flags


def sem_mlp_backward(mlp, feats, labels, class_w, want_loss=True, stream=None):
    n = feats.shape[0]
    _f32(feats, (n, 136))
    cw = np.ascontiguousarray(np.asarray(class_w, dtype=np.float32))
    loss = C.c_double(0.0)
    _check(LIB.sem_mlp_backward(mlp.h, _ptr(feats), _ptr(labels), _ptr(cw), n,
                                C.byref(loss) if want_loss else None, _stream(stream)))
    return loss.value if want_loss else None


def sem_mlp_adam(mlp, lr, stream=None):
    _check(LIB.sem_mlp_adam(mlp.h, float(lr), _stream(stream)))


def sem_checkpoint_write(mesh, q, path, time=0.0, step=0, stream=None):
    _f64(q, mesh.field_shape)
    _check(LIB.sem_checkpoint_write(mesh.h, _ptr(q), float(time), int(step), str(path).encode(),
                                    _stream(stream)))


def sem_checkpoint_read_mesh(path):
    """(mesh, time, step) from a checkpoint file (host only)."""
    h = C.c_void_p()
    t = C.c_double(0.0)
    s = C.c_longlong(0)
    _check(LIB.sem_checkpoint_read_mesh(str(path).encode(), C.byref(h), C.byref(t), C.byref(s)))
    return Mesh(h.value), t.value, s.value


def sem_checkpoint_read_state(path, mesh, q, stream=None):
    _f64(q, mesh.field_shape)
    _check(LIB.sem_checkpoint_read_state(str(path).encode(), mesh.h, _ptr(q), _stream(stream)))
    return q


def sem_selftest_device_once(n_devices, n_threads):
    """Host-only check of the per-device one-time set-up: how many times the
    set-up ran for each simulated device ordinal (1 each when correct)."""
    out = (C.c_int * n_devices)()
    _check(LIB.sem_selftest_device_once(n_devices, n_threads, out))
    return list(out)


def sem_peak_probe(precision, stream=None):
    """float32 (SEM_PREC_MIXED) or float64 (SEM_PREC_FP64) FMA rate, TFLOP/s."""
    out = C.c_double()
    _check(LIB.sem_peak_probe(precision, C.byref(out), _stream(stream)))
    return out.value


def sem_mlp_select_forward(mlp, tc):
    """1: tcgen05 tensor-core forward (default), 0: mma.sync forward."""
    _check(LIB.sem_mlp_select_forward(mlp.h, int(tc)))


def sem_mlp_status(mlp, stream=None):
    out = C.c_int()
    _check(LIB.sem_mlp_status(mlp.h, C.byref(out), _stream(stream)))
    return out.value
