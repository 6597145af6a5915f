"""Python binding of libnif (include/nif.h): argument marshalling only.

Every function named ``nif_*`` here calls the C entry point of the same name;
torch tensors are used only as device memory (their data pointers are passed
through) and torch streams as CUDA streams. All computation happens in the
library's CUDA kernels. If libnif.so is missing the import fails loudly: there
is no CPU or eager fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# NIF_BOUNDS_BUILD=1 loads the bounds-checked build of the same sources
# (build(bounds=True): index checks that count failures instead of trapping)
LIB_PATH = os.path.join(_HERE, "libnif_bounds.so" if os.environ.get("NIF_BOUNDS_BUILD") == "1" else "libnif.so")

NIF_OK, NIF_ERR_ARG, NIF_ERR_CUDA, NIF_ERR_OOM, NIF_ERR_CAPACITY, NIF_ERR_TIMEOUT, NIF_ERR_NAN, NIF_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6, -7
NIF_FP32, NIF_BF16, NIF_FP16 = 0, 1, 2
NIF_PARAM_TABLES, NIF_PARAM_LOGVAR, NIF_PARAM_LAYER0 = 0, 1, 16
NIF_SHADOW_ONLY = 1
NIF_FLAG_FIXED_TASK_WEIGHTS, NIF_FLAG_SIGMOID_DISTANCE, NIF_FLAG_MIXED_TRAINING = 1, 2, 4
NIF_FLAG_CONCAT_ENCODING = 8
NIF_FLAG_BILINEAR_FACES = 16
NIF_KNOB_WAIT_NS, NIF_KNOB_SEG_SCRATCH, NIF_KNOB_QUERY_SEGS, NIF_KNOB_BATCH_AT, NIF_KNOB_FP32_FUSED = 1, 2, 3, 4, 5
NIF_KNOB_QUERY_FUSED, NIF_KNOB_STEP_PRIORITY, NIF_KNOB_DEFER_WEIGHTS = 6, 7, 8
NIF_KNOB_STEP_FWD_CTAS = 9
NIF_KNOB_STEP_BWD_CTAS = 10
NIF_KNOB_DETERMINISTIC = 11
NIF_KNOB_ORDER_BITS = 12
NIF_KNOB_FAIL_ALLOC = 13
NIF_KNOB_BWD_SPLIT = 14
NIF_PROBE_RED8, NIF_PROBE_RED16, NIF_PROBE_LOAD8, NIF_PROBE_LOAD4 = 1, 2, 3, 4
NIF_PROBE_RED8_WARP, NIF_PROBE_RED16_WARP, NIF_PROBE_LOAD8_WARP, NIF_PROBE_LOAD4_WARP = 5, 6, 7, 8

_STATUS = {0: "NIF_OK", -1: "NIF_ERR_ARG", -2: "NIF_ERR_CUDA", -3: "NIF_ERR_OOM", -4: "NIF_ERR_CAPACITY",
           -5: "NIF_ERR_TIMEOUT", -6: "NIF_ERR_NAN", -7: "NIF_ERR_STATE"}
_TORCH_DT = {NIF_FP32: torch.float32, NIF_BF16: torch.bfloat16, NIF_FP16: torch.float16}


class NifError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class nif_config(ctypes.Structure):
    _fields_ = [("voxel_res", ctypes.c_int), ("pe_bands", ctypes.c_int), ("levels", ctypes.c_int),
                ("feats", ctypes.c_int), ("log2_table", ctypes.c_int), ("base_res", ctypes.c_int),
                ("growth", ctypes.c_float), ("mlp_depth", ctypes.c_int), ("mlp_width", ctypes.c_int),
                ("n_materials", ctypes.c_int), ("precision", ctypes.c_int), ("flags", ctypes.c_uint),
                ("seed", ctypes.c_ulonglong)]


class nif_mesh(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("n_verts", ctypes.c_int), ("tris", ctypes.c_void_p),
                ("n_tris", ctypes.c_int), ("tri_albedo", ctypes.c_void_p), ("tri_material", ctypes.c_void_p)]


class nif_pose(ctypes.Structure):
    _fields_ = [("bend", ctypes.c_float), ("twist", ctypes.c_float), ("taper", ctypes.c_float)]


# structured views of the 16/32-byte records, for reading results back
SEGMENT_DTYPE = np.dtype([("ray", np.uint32), ("voxel", np.uint32), ("t0", np.float32), ("t1", np.float32)])
LINSEG_DTYPE = np.dtype([("p0", np.float32, 3), ("p1", np.float32, 3), ("l_def", np.float32), ("l_rest", np.float32)])
LABEL_DTYPE = np.dtype([("tpar", np.float32), ("normal", np.float32, 3), ("albedo", np.float32, 3), ("occ", np.uint8),
                        ("material", np.uint8), ("pad", np.uint8, 2)])
HIT_DTYPE = np.dtype([("D", np.float32), ("n", np.float32, 3), ("albedo", np.float32, 3), ("hit", np.uint8),
                      ("material", np.uint8), ("pad", np.uint8, 2)])

_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def lib() -> ctypes.CDLL:
    """Load libnif.so (built by paper_2604_24666_gb300.build); never falls back."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); "
                              "run paper_2604_24666_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "nif_create": ([ctypes.POINTER(nif_config), ctypes.POINTER(nif_mesh), ctypes.POINTER(_vp)], ctypes.c_int),
            "nif_destroy": ([_vp], None),
            "nif_last_error": ([_vp], ctypes.c_char_p),
            "nif_param_bytes": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
            "nif_get_params": ([_vp, ctypes.c_int, _vp, ctypes.c_size_t], ctypes.c_int),
            "nif_set_params": ([_vp, ctypes.c_int, _vp, ctypes.c_size_t], ctypes.c_int),
            "nif_get_grad": ([_vp, ctypes.c_int, _vp, ctypes.c_size_t], ctypes.c_int),
            "nif_set_grad": ([_vp, ctypes.c_int, _vp, ctypes.c_size_t], ctypes.c_int),
            "nif_zero_grad": ([_vp, _vp], ctypes.c_int),
            "nif_reset_optimizer": ([_vp], ctypes.c_int),
            "nif_adam_step": ([_vp, ctypes.c_float, ctypes.c_float, _vp], ctypes.c_int),
            "nif_get_voxels": ([_vp, _vp, _vp, _vp, _i64, ctypes.POINTER(_i64)], ctypes.c_int),
            "nif_segments": ([_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp, _i64, ctypes.POINTER(_i64),
                              _vp], ctypes.c_int),
            "nif_linearize": ([_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _i64, _vp, _vp], ctypes.c_int),
            "nif_encode_points": ([_vp, _vp, _i64, _vp, ctypes.c_int, _vp, _vp], ctypes.c_int),
            "nif_encode_segments": ([_vp, _vp, _i64, _vp, ctypes.c_int, ctypes.c_int, _vp], ctypes.c_int),
            "nif_encode_points_backward": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp], ctypes.c_int),
            "nif_encode_segments_backward": ([_vp, _vp, _i64, _vp, _vp, _vp], ctypes.c_int),
            "nif_pose_gradient": ([_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp], ctypes.c_int),
            "nif_mlp_forward": ([_vp, _vp, ctypes.c_int, _i64, _vp, ctypes.c_int, _vp, _vp], ctypes.c_int),
            "nif_mlp_backward": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp], ctypes.c_int),
            "nif_mlp_backward_lowp": ([_vp, _vp, ctypes.c_int, _i64, _vp, _vp, _vp], ctypes.c_int),
            "nif_loss_scale": ([_vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "nif_set_loss_scale": ([_vp, ctypes.c_float], ctypes.c_int),
            "nif_adam_step_scaled": ([_vp, ctypes.c_float, ctypes.c_float, _vp], ctypes.c_int),
            "nif_pose_step": ([_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _i64, _vp, _vp, _vp], ctypes.c_int),
            "nif_shadow_rays": ([_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_float, ctypes.c_float, _vp, _vp],
                                ctypes.c_int),
            "nif_labels": ([_vp, _vp, _vp, _i64, _vp, _vp], ctypes.c_int),
            "nif_loss": ([_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp], ctypes.c_int),
            "nif_reconstruct": ([_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp,
                                 ctypes.c_uint, _vp], ctypes.c_int),
            "nif_query": ([_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, ctypes.c_uint, _vp], ctypes.c_int),
            "nif_train_step_rays": ([_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _i64, ctypes.c_float,
                                     ctypes.c_float, _vp, _vp], ctypes.c_int),
            "nif_train_step": ([_vp, _i64, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_float, ctypes.c_float, _vp, _vp,
                                _vp], ctypes.c_int),
            "nif_train_steps": ([_vp, ctypes.c_int, _i64, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_float, ctypes.c_float,
                                 _vp, _vp], ctypes.c_int),
            "nif_train_steps_rays": ([_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _i64, ctypes.c_float,
                                      ctypes.c_float, _vp, _vp], ctypes.c_int),
            "nif_sample_rays": ([_vp, ctypes.c_ulonglong, ctypes.c_int, ctypes.c_int, _vp, _vp], ctypes.c_int),
            "nif_segments_noalloc": ([_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp, _i64,
                                      ctypes.POINTER(_i64), _vp], ctypes.c_int),
            "nif_segments_walk": ([_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp, _i64,
                                   ctypes.POINTER(_i64), ctypes.c_uint, _vp], ctypes.c_int),
            "nif_query_plan_create": ([_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _i64, ctypes.c_uint,
                                       ctypes.c_int, _vp, ctypes.POINTER(_vp)], ctypes.c_int),
            "nif_query_plan_run": ([_vp, _vp, _vp], ctypes.c_int),
            "nif_query_plan_info": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_i64), ctypes.POINTER(_i64)],
                                    ctypes.c_int),
            "nif_query_plan_destroy": ([_vp], None),
            "nif_sync_status": ([_vp, _vp], ctypes.c_int),
            "nif_set_knob": ([_vp, ctypes.c_int, ctypes.c_double], ctypes.c_int),
            "nif_probe_memory": ([_vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), _vp], ctypes.c_int),
            "nif_encoder_points": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)], ctypes.c_int),
            "nif_set_field": ([_vp, ctypes.c_int, ctypes.c_int, _vp], ctypes.c_int),
            "nif_get_field": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _vp, ctypes.c_size_t],
                              ctypes.c_int),
            "nif_field_gradient": ([_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _i64, _vp, _vp, _vp], ctypes.c_int),
            "nif_field_step": ([_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _i64, _vp, ctypes.c_float,
                                ctypes.c_float, ctypes.c_float, _vp, _vp], ctypes.c_int),
            "nif_checkpoint_bytes": ([_vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
            "nif_checkpoint_save": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
            "nif_checkpoint_load": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
            "nif_kernel_launches": ([], ctypes.c_ulonglong),
            "nif_bounds_check": ([ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_ulonglong)], ctypes.c_int),
            "nif_profile": ([_vp, ctypes.c_int], ctypes.c_int),
            "nif_profile_filter": ([_vp, ctypes.c_char_p], ctypes.c_int),
            "nif_profile_timeline": ([_vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "nif_profile_read": ([_vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    """Names of the entry points this binding resolves (all must exist)."""
    lib()
    return sorted(n for n in dir(_lib) if n.startswith("nif_"))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return t


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _poses(poses):
    p = np.ascontiguousarray(np.asarray(poses, np.float32).reshape(-1, 3))
    arr = (nif_pose * len(p))()
    for i, (b, t, a) in enumerate(p):
        arr[i] = nif_pose(float(b), float(t), float(a))
    return arr, len(p)


def _check(h, st):
    if st != NIF_OK:
        msg = lib().nif_last_error(h.value if isinstance(h, ctypes.c_void_p) else h)
        raise NifError(st, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# C-ABI functions (same names)
# ---------------------------------------------------------------------------

def make_config(net, precision=NIF_FP32, seed=0, flags=0) -> nif_config:
    if getattr(net, "encoding", "composed") == "concat":
        flags |= NIF_FLAG_CONCAT_ENCODING
    if getattr(net, "faces", "triangles") == "bilinear":
        flags |= NIF_FLAG_BILINEAR_FACES
    return nif_config(net.voxel_res, net.pe_bands, net.levels, net.feats, net.log2_table, net.base_res,
                      float(net.growth), net.mlp_depth, net.mlp_width, net.n_materials, int(precision), int(flags),
                      int(seed))


def nif_create(net, mesh, precision=NIF_FP32, seed=0, flags=0):
    cfg = make_config(net, precision, seed, flags)
    v = np.ascontiguousarray(mesh.verts, np.float32)
    t = np.ascontiguousarray(mesh.tris, np.int32)
    a = np.ascontiguousarray(mesh.albedo, np.float32)
    m = np.ascontiguousarray(mesh.material, np.uint8)
    cm = nif_mesh(v.ctypes.data, len(v), t.ctypes.data, len(t), a.ctypes.data, m.ctypes.data)
    h = ctypes.c_void_p()
    st = lib().nif_create(ctypes.byref(cfg), ctypes.byref(cm), ctypes.byref(h))
    if st != NIF_OK:
        raise NifError(st, lib().nif_last_error(None).decode())
    return h


def nif_destroy(h):
    lib().nif_destroy(h)


def nif_param_bytes(h, group) -> int:
    n = ctypes.c_size_t()
    _check(h, lib().nif_param_bytes(h, group, ctypes.byref(n)))
    return n.value


def nif_get_params(h, group) -> np.ndarray:
    out = np.zeros(nif_param_bytes(h, group) // 4, np.float32)
    _check(h, lib().nif_get_params(h, group, _ptr(out), out.nbytes))
    return out


def nif_set_params(h, group, arr):
    a = np.ascontiguousarray(arr, np.float32).reshape(-1)
    _check(h, lib().nif_set_params(h, group, _ptr(a), a.nbytes))


def nif_get_grad(h, group) -> np.ndarray:
    out = np.zeros(nif_param_bytes(h, group) // 4, np.float32)
    _check(h, lib().nif_get_grad(h, group, _ptr(out), out.nbytes))
    return out


def nif_set_grad(h, group, arr):
    a = np.ascontiguousarray(arr, np.float32).reshape(-1)
    _check(h, lib().nif_set_grad(h, group, _ptr(a), a.nbytes))


def nif_zero_grad(h, stream=None):
    _check(h, lib().nif_zero_grad(h, _stream(stream)))


def nif_reset_optimizer(h):
    _check(h, lib().nif_reset_optimizer(h))


def nif_adam_step(h, lr_grid, lr_mlp, stream=None):
    _check(h, lib().nif_adam_step(h, lr_grid, lr_mlp, _stream(stream)))


def nif_get_voxels(h, N):
    occ = np.zeros(N ** 3, np.uint8)
    ptr = np.zeros(N ** 3 + 1, np.int64)
    n = _i64()
    _check(h, lib().nif_get_voxels(h, _ptr(occ), _ptr(ptr), None, 0, ctypes.byref(n)))
    idx = np.zeros(max(n.value, 1), np.int32)
    _check(h, lib().nif_get_voxels(h, _ptr(occ), _ptr(ptr), _ptr(idx), n.value, None))
    return occ, ptr, idx[:n.value]


def nif_segments(h, poses, rays, inst_offsets=None, seg_cap=None, stream=None):
    """rays: cuda float32 [n, 8]. Returns (ray_offsets [n+1] int32-as-uint32, segs [S, 4] raw)."""
    p, n_inst = _poses(poses)
    n = rays.shape[0]
    offs = torch.zeros(n + 1, dtype=torch.int32, device=rays.device)
    if seg_cap is None:      # count-only pass first
        total = _i64()
        _check(h, lib().nif_segments(h, p, n_inst, _ptr(rays), _ptr(inst_offsets), n, _ptr(offs), None, 0,
                                     ctypes.byref(total), _stream(stream)))
        seg_cap = max(1, total.value)
    segs = torch.zeros((seg_cap, 4), dtype=torch.int32, device=rays.device)
    total = _i64()
    _check(h, lib().nif_segments(h, p, n_inst, _ptr(rays), _ptr(inst_offsets), n, _ptr(offs), _ptr(segs), seg_cap,
                                 ctypes.byref(total), _stream(stream)))
    return offs, segs[:total.value]


NIF_WALK_FIRST_HIT = 1


def nif_segments_walk(h, poses, rays, inst_offsets=None, seg_cap=None, flags=0, stream=None):
    """Segments by BVH first hit + exit-face walk (same outputs as nif_segments).
    flags=NIF_WALK_FIRST_HIT: only the first BVH query; returns (ray_offsets, None)."""
    p, n_inst = _poses(poses)
    n = rays.shape[0]
    offs = torch.zeros(n + 1, dtype=torch.int32, device=rays.device)
    total = _i64()
    if seg_cap is None or flags:
        _check(h, lib().nif_segments_walk(h, p, n_inst, _ptr(rays), _ptr(inst_offsets), n, _ptr(offs), None, 0,
                                          ctypes.byref(total), flags, _stream(stream)))
        if flags:
            return offs, None
        seg_cap = max(1, total.value)
    segs = torch.zeros((seg_cap, 4), dtype=torch.int32, device=rays.device)
    _check(h, lib().nif_segments_walk(h, p, n_inst, _ptr(rays), _ptr(inst_offsets), n, _ptr(offs), _ptr(segs),
                                      seg_cap, ctypes.byref(total), flags, _stream(stream)))
    return offs, segs[:total.value]


def nif_segments_noalloc(h, poses, rays, ray_offsets, segs, inst_offsets=None, stream=None):
    """Allocation-free segments into the caller's ray_offsets [n+1] and segs [cap, 4] (None: count only);
    returns the total."""
    p, n_inst = _poses(poses)
    total = _i64()
    cap = segs.shape[0] if segs is not None else 0
    _check(h, lib().nif_segments_noalloc(h, p, n_inst, _ptr(rays), _ptr(inst_offsets), rays.shape[0],
                                         _ptr(ray_offsets), _ptr(segs), cap, ctypes.byref(total),
                                         _stream(stream)))
    return total.value


def nif_linearize(h, poses, rays, segs, inst_offsets=None, stream=None):
    p, n_inst = _poses(poses)
    lin = torch.zeros((segs.shape[0], 8), dtype=torch.float32, device=rays.device)
    _check(h, lib().nif_linearize(h, p, n_inst, _ptr(rays), _ptr(inst_offsets), rays.shape[0], _ptr(segs),
                                  segs.shape[0], _ptr(lin), _stream(stream)))
    return lin


def nif_encode_points(h, pts, width, out_dtype=NIF_FP32, rows=False, n_terms=None, levels=None, stream=None):
    n = pts.shape[0]
    feats = torch.zeros((n, width), dtype=_TORCH_DT[out_dtype], device=pts.device)
    r = torch.zeros((n, n_terms * levels), dtype=torch.int32, device=pts.device) if rows else None
    _check(h, lib().nif_encode_points(h, _ptr(pts), n, _ptr(feats), out_dtype, _ptr(r), _stream(stream)))
    return feats, r


def nif_encode_segments(h, lin, in_dim, out_dtype=NIF_FP32, table_dtype=NIF_FP32, stream=None):
    feats = torch.zeros((lin.shape[0], in_dim), dtype=_TORCH_DT[out_dtype], device=lin.device)
    _check(h, lib().nif_encode_segments(h, _ptr(lin), lin.shape[0], _ptr(feats), out_dtype, table_dtype,
                                        _stream(stream)))
    return feats


def nif_encode_points_backward(h, pts, dfeats, dtables=None, want_dpts=True, stream=None):
    """dtables None accumulates into the handle's own gradient buffer."""
    dpts = torch.zeros_like(pts) if want_dpts else None
    _check(h, lib().nif_encode_points_backward(h, _ptr(pts), pts.shape[0], _ptr(dfeats), _ptr(dtables), _ptr(dpts),
                                               _stream(stream)))
    return dpts


def nif_encode_segments_backward(h, lin, dfeats, dtables, stream=None):
    _check(h, lib().nif_encode_segments_backward(h, _ptr(lin), lin.shape[0], _ptr(dfeats), _ptr(dtables),
                                                 _stream(stream)))


def nif_pose_gradient(h, poses, segs, lin, dfeats, inst_offsets=None, want_dp=False, stream=None):
    """dL/d(bend, twist, taper) [n_inst, 3] of sum(dfeats * features) for fixed deformed end points."""
    p, n_inst = _poses(poses)
    dposes = torch.zeros((n_inst, 3), dtype=torch.float32, device=lin.device)
    dp = torch.zeros((lin.shape[0], 6), dtype=torch.float32, device=lin.device) if want_dp else None
    _check(h, lib().nif_pose_gradient(h, p, n_inst, _ptr(inst_offsets), _ptr(segs), _ptr(lin), lin.shape[0],
                                      _ptr(dfeats), _ptr(dposes), _ptr(dp), _stream(stream)))
    return (dposes, dp) if want_dp else dposes


def nif_mlp_forward(h, x, precision=NIF_FP32, acts=None, stream=None):
    xdt = {torch.float32: NIF_FP32, torch.bfloat16: NIF_BF16, torch.float16: NIF_FP16}[x.dtype]
    out = torch.zeros((x.shape[0], 16), dtype=torch.float32, device=x.device)
    _check(h, lib().nif_mlp_forward(h, _ptr(x), xdt, x.shape[0], _ptr(out), precision, _ptr(acts), _stream(stream)))
    return out


def nif_mlp_backward(h, x, acts, dout, want_dx=True, stream=None):
    dx = torch.zeros_like(x) if want_dx else None
    _check(h, lib().nif_mlp_backward(h, _ptr(x), x.shape[0], _ptr(acts), _ptr(dout), _ptr(dx), _stream(stream)))
    return dx


def nif_mlp_backward_lowp(h, x, dout, want_dx=True, stream=None):
    """Tensor-core MLP backward of the mixed path: x [n][in_dim] BF16/FP16
    (the handle's precision), dout [n][16] FP32. Adds S * dL/dW into the
    gradient buffer and returns S * dL/dx (FP32) with S the loss scale."""
    dt = {torch.bfloat16: NIF_BF16, torch.float16: NIF_FP16}[x.dtype]
    dx = torch.zeros((x.shape[0], x.shape[1]), dtype=torch.float32, device=x.device) if want_dx else None
    _check(h, lib().nif_mlp_backward_lowp(h, _ptr(x), dt, x.shape[0], _ptr(dout), _ptr(dx), _stream(stream)))
    return dx


def nif_loss_scale(h):
    """(S, skipped steps) of the mixed-precision path."""
    sc, sk = ctypes.c_float(), ctypes.c_int()
    _check(h, lib().nif_loss_scale(h, ctypes.byref(sc), ctypes.byref(sk)))
    return sc.value, sk.value


def nif_set_loss_scale(h, scale):
    _check(h, lib().nif_set_loss_scale(h, float(scale)))


def nif_adam_step_scaled(h, lr_grid, lr_mlp, stream=None):
    _check(h, lib().nif_adam_step_scaled(h, lr_grid, lr_mlp, _stream(stream)))


def nif_pose_step(h, poses, rays, n_segments, inst_offsets=None, want_loss=False, dposes=None, stream=None):
    """dL/d(bend, twist, taper) [n_inst, 3] of the task loss on the segments of `rays`
    (tables, weights and s fixed); returns (dposes, loss parts or None)."""
    p, n_inst = _poses(poses)
    if dposes is None:
        dposes = torch.zeros((n_inst, 3), dtype=torch.float32, device=rays.device)
    parts = np.zeros(6, np.float64) if want_loss else None
    _check(h, lib().nif_pose_step(h, p, n_inst, _ptr(rays), _ptr(inst_offsets), rays.shape[0], int(n_segments),
                                  _ptr(dposes), _ptr(parts), _stream(stream)))
    return dposes, parts


def nif_shadow_rays(h, rays, hits, light_dir, eps=1e-4, tmax=4.0, out=None, stream=None):
    """Shadow rays [n, 8] from primary rays and their hits toward a directional light."""
    if out is None:
        out = torch.empty_like(rays)
    L = (ctypes.c_float * 3)(*[float(v) for v in light_dir])
    _check(h, lib().nif_shadow_rays(h, _ptr(rays), _ptr(hits), rays.shape[0], ctypes.cast(L, ctypes.c_void_p),
                                    float(eps), float(tmax),
                                    _ptr(out), _stream(stream)))
    return out


def nif_labels(h, segs, lin, stream=None):
    lab = torch.zeros((segs.shape[0], 8), dtype=torch.float32, device=segs.device)
    _check(h, lib().nif_labels(h, _ptr(segs), _ptr(lin), segs.shape[0], _ptr(lab), _stream(stream)))
    return lab


def nif_loss(h, out, labels, lin, want_dout=True, stream=None):
    dout = torch.zeros_like(out) if want_dout else None
    parts = np.zeros(6, np.float64)
    _check(h, lib().nif_loss(h, _ptr(out), _ptr(labels), _ptr(lin), out.shape[0], _ptr(dout), _ptr(parts),
                             _stream(stream)))
    return parts, dout


def nif_reconstruct(h, poses, rays, ray_offsets, segs, lin, out, inst_offsets=None, flags=0, stream=None):
    p, n_inst = _poses(poses)
    hits = torch.zeros((rays.shape[0], 8), dtype=torch.float32, device=rays.device)
    _check(h, lib().nif_reconstruct(h, p, n_inst, _ptr(rays), _ptr(inst_offsets), rays.shape[0], _ptr(ray_offsets),
                                    _ptr(segs), _ptr(lin), _ptr(out), _ptr(hits), flags, _stream(stream)))
    return hits


def nif_query(h, poses, rays, inst_offsets=None, flags=0, hits=None, stream=None):
    p, n_inst = _poses(poses)
    if hits is None:
        hits = torch.zeros((rays.shape[0], 8), dtype=torch.float32, device=rays.device)
    _check(h, lib().nif_query(h, p, n_inst, _ptr(rays), _ptr(inst_offsets), rays.shape[0], _ptr(hits), flags,
                              _stream(stream)))
    return hits


def nif_train_step_rays(h, poses, rays, n_segments, inst_offsets=None, lr_grid=1e-2, lr_mlp=1e-3, want_loss=True,
                        stream=None):
    p, n_inst = _poses(poses)
    loss = np.zeros(6, np.float64) if want_loss else None
    _check(h, lib().nif_train_step_rays(h, p, n_inst, _ptr(rays), _ptr(inst_offsets), rays.shape[0], n_segments,
                                        lr_grid, lr_mlp, _ptr(loss), _stream(stream)))
    return loss


def nif_train_steps(h, n_steps, n_segments, n_poses, first_seed, lr_grid=1e-2, lr_mlp=5e-3, want_loss=False,
                    stream=None):
    """n_steps training steps with seeds first_seed.. (the next batch built beside each step);
    returns the last step's loss parts [6] when want_loss."""
    loss = np.zeros(6, np.float64) if want_loss else None
    _check(h, lib().nif_train_steps(h, n_steps, n_segments, n_poses, first_seed, lr_grid, lr_mlp, _ptr(loss),
                                    _stream(stream)))
    return loss


def nif_train_steps_rays(h, poses, rays_host, n_segments, inst_offsets=None, lr_grid=1e-2, lr_mlp=1e-3,
                         want_loss=True, stream=None):
    """len(rays_host) training steps; step i on the rays rays_host[i] (a CPU tensor
    [n_steps, n_rays, 8], pinned for overlap) and the poses poses[i] ([n_steps, n_inst, 3]);
    returns every step's loss parts [n_steps, 6] when want_loss."""
    assert rays_host.device.type == "cpu" and rays_host.dim() == 3 and rays_host.shape[2] == 8
    n_steps, n_rays = rays_host.shape[0], rays_host.shape[1]
    pa = np.asarray(poses, np.float32).reshape(n_steps, -1, 3)
    p, _ = _poses(pa)
    rays_host = rays_host.contiguous()
    loss = np.zeros((n_steps, 6), np.float64) if want_loss else None
    _check(h, lib().nif_train_steps_rays(h, n_steps, p, pa.shape[1], _ptr(rays_host), _ptr(inst_offsets), n_rays,
                                         n_segments, lr_grid, lr_mlp, _ptr(loss), _stream(stream)))
    return loss


def nif_train_step(h, n_segments, n_poses, step_seed, lr_grid=1e-2, lr_mlp=1e-3, want_loss=True, stream=None):
    loss = np.zeros(6, np.float64) if want_loss else None
    poses = (nif_pose * n_poses)()
    _check(h, lib().nif_train_step(h, n_segments, n_poses, step_seed, lr_grid, lr_mlp, poses, _ptr(loss),
                                   _stream(stream)))
    return loss, np.array([[q.bend, q.twist, q.taper] for q in poses], np.float32)


def nif_sample_rays(h, step_seed, stream_id, n, device="cuda", stream=None):
    rays = torch.zeros((n, 8), dtype=torch.float32, device=device)
    _check(h, lib().nif_sample_rays(h, step_seed, stream_id, n, _ptr(rays), _stream(stream)))
    return rays


class QueryPlan:
    """A captured batched query (nif_query_plan_*); buffers stay bound to it."""

    def __init__(self, h, poses, rays, hits, inst_offsets=None, seg_capacity=0, flags=0, autotune=True):
        p, n_inst = _poses(poses)
        self.h = h
        self.n_inst = n_inst
        self._keep = (rays, hits, inst_offsets)
        out = ctypes.c_void_p()
        _check(h, lib().nif_query_plan_create(h, n_inst, _ptr(rays), _ptr(inst_offsets), rays.shape[0], _ptr(hits),
                                              int(seg_capacity), flags, int(autotune), p, ctypes.byref(out)))
        self.p = out

    def run(self, poses, stream=None):
        p, n_inst = _poses(poses)
        if n_inst != self.n_inst:
            raise ValueError("pose count differs from the plan's")
        _check(self.h, lib().nif_query_plan_run(self.p, p, _stream(stream)))

    def info(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        d, e = _i64(), _i64()
        _check(self.h, lib().nif_query_plan_info(self.p, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                                 ctypes.byref(d), ctypes.byref(e)))
        return dict(trav_warps=a.value, enc_threads=b.value, enc_blocks_per_sm=c.value, tc_chunk=d.value,
                    seg_capacity=e.value)

    def close(self):
        if self.p:
            lib().nif_query_plan_destroy(self.p)
            self.p = None


def nif_sync_status(h, stream=None):
    _check(h, lib().nif_sync_status(h, _stream(stream)))


def nif_set_field(h, delta):
    """Learned deformation field: delta [n_inst, G, G, G, 3] float32 (index
    [i][c][b][a] of node (a, b, c)/(G-1)); None or an empty array removes it."""
    if delta is None or np.size(delta) == 0:
        _check(h, lib().nif_set_field(h, 0, 0, None))
        return
    d = np.ascontiguousarray(delta, np.float32)
    assert d.ndim == 5 and d.shape[1] == d.shape[2] == d.shape[3] and d.shape[4] == 3
    _check(h, lib().nif_set_field(h, d.shape[0], d.shape[1], _ptr(d)))


def nif_get_field(h):
    """The field [n_inst, G, G, G, 3] float32 (None without one)."""
    n, G = ctypes.c_int(0), ctypes.c_int(0)
    _check(h, lib().nif_get_field(h, ctypes.byref(n), ctypes.byref(G), None, 0))
    if n.value == 0:
        return None
    d = np.zeros((n.value, G.value, G.value, G.value, 3), np.float32)
    _check(h, lib().nif_get_field(h, None, None, _ptr(d), d.nbytes))
    return d


def nif_field_gradient(h, poses, segs, lin, dfeats, inst_offsets=None, stream=None):
    """d/d(field) [n_inst, G, G, G, 3] of sum(dfeats * features) for fixed deformed end points."""
    p, n_inst = _poses(poses)
    n_f, G = ctypes.c_int(0), ctypes.c_int(0)
    _check(h, lib().nif_get_field(h, ctypes.byref(n_f), ctypes.byref(G), None, 0))
    out = torch.zeros((max(n_f.value, 1), G.value, G.value, G.value, 3), dtype=torch.float32, device=lin.device)
    _check(h, lib().nif_field_gradient(h, p, n_inst, _ptr(inst_offsets), _ptr(segs), _ptr(lin), lin.shape[0],
                                       _ptr(dfeats), _ptr(out), _stream(stream)))
    return out


def nif_field_step(h, poses, rays, n_segments, target_poses, inst_offsets=None, lr_field=1e-3, lr_grid=0.0,
                   lr_mlp=0.0, want_loss=True, stream=None):
    """One fitting step of the field towards the target poses' deformation; returns the loss parts."""
    p, n_inst = _poses(poses)
    t, n_t = _poses(target_poses)
    assert n_t == n_inst
    loss = np.zeros(6, np.float64) if want_loss else None
    _check(h, lib().nif_field_step(h, p, n_inst, _ptr(rays), _ptr(inst_offsets), rays.shape[0], n_segments, t,
                                   lr_field, lr_grid, lr_mlp, _ptr(loss), _stream(stream)))
    return loss


def nif_probe_memory(h, kind, buf, iters=64, stream=None):
    """(GB/s of payload, ms per launch) of one memory pattern over the device buffer buf."""
    g, ms = ctypes.c_double(0), ctypes.c_double(0)
    _check(h, lib().nif_probe_memory(h, kind, _ptr(buf), buf.numel() * buf.element_size(), iters, ctypes.byref(g),
                                     ctypes.byref(ms), _stream(stream)))
    return g.value, ms.value


def nif_encoder_points(h):
    """(distinct end points, segments) of the handle's last segment encoding."""
    a, b = _i64(0), _i64(0)
    _check(h, lib().nif_encoder_points(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def nif_set_knob(h, knob, value):
    """Set one of the handle's NIF_KNOB_* tuning knobs (include/nif.h gives
    each one's values). Knobs choose schedules, kernels or scratch sizes,
    not results. Examples: NIF_KNOB_WAIT_NS bounds the tensor-core kernels'
    waits (ns; 0 = default), NIF_KNOB_SEG_SCRATCH scales the single-traversal
    segment scratch, and NIF_KNOB_STEP_FWD_CTAS / NIF_KNOB_STEP_BWD_CTAS set
    how the FP32 training step shares SMs between concurrent kernels.
    NIF_KNOB_DETERMINISTIC = 1 is the one knob that changes results (in
    their last bits): gradients are then summed in an order-free way, so
    that repeated runs and resumed checkpoints give bit-identical states."""
    _check(h, lib().nif_set_knob(h, knob, float(value)))


def nif_checkpoint_save(h) -> bytes:
    n = ctypes.c_size_t()
    _check(h, lib().nif_checkpoint_bytes(h, ctypes.byref(n)))
    buf = (ctypes.c_uint8 * n.value)()
    _check(h, lib().nif_checkpoint_save(h, ctypes.cast(buf, ctypes.c_void_p), n.value))
    return bytes(buf)


def nif_checkpoint_load(h, blob: bytes):
    buf = (ctypes.c_uint8 * len(blob)).from_buffer_copy(blob)
    _check(h, lib().nif_checkpoint_load(h, ctypes.cast(buf, ctypes.c_void_p), len(blob)))


def nif_bounds_check():
    """(enabled, failures): whether this is the bounds-checked build, and the
    index checks that failed since the last call (then cleared)."""
    en, n = ctypes.c_int(), ctypes.c_ulonglong()
    st = lib().nif_bounds_check(ctypes.byref(en), ctypes.byref(n))
    if st != NIF_OK:
        raise NifError(st, "nif_bounds_check failed")
    return bool(en.value), int(n.value)


def nif_kernel_launches() -> int:
    return int(lib().nif_kernel_launches())


def nif_profile(h, enable):
    _check(h, lib().nif_profile(h, int(enable)))


def nif_profile_filter(h, names=None):
    """Time only the named stages (an iterable of names, or None for all)."""
    arg = ",".join(names).encode() if names else None
    _check(h, lib().nif_profile_filter(h, arg))


def nif_profile_timeline(h):
    """[(stage, start ms, end ms)] of the timed stages in launch order, relative
    to the first one's start (read before nif_profile_read folds them)."""
    n = ctypes.c_int()
    _check(h, lib().nif_profile_timeline(h, -1, None, 0, None, None, ctypes.byref(n)))
    out = []
    for i in range(n.value):
        name = ctypes.create_string_buffer(64)
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(h, lib().nif_profile_timeline(h, i, name, 64, ctypes.byref(a), ctypes.byref(b), None))
        out.append((name.value.decode(), a.value, b.value))
    return out


def nif_profile_read(h):
    """{stage: (total ms, timed launches)} of the handle's profiling record."""
    n = ctypes.c_int()
    _check(h, lib().nif_profile_read(h, -1, None, 0, None, None, ctypes.byref(n)))
    out = {}
    for i in range(n.value):
        name = ctypes.create_string_buffer(64)
        ms = ctypes.c_double()
        cnt = ctypes.c_long()
        _check(h, lib().nif_profile_read(h, i, name, 64, ctypes.byref(ms), ctypes.byref(cnt), None))
        out[name.value.decode()] = (ms.value, cnt.value)
    return out


# ---------------------------------------------------------------------------
# Convenience owner of a handle
# ---------------------------------------------------------------------------

class Nif:
    """Owns a nif_handle for one shape and configuration (see synth.NetConfig)."""

    def __init__(self, net, mesh, precision=NIF_FP32, seed=0, flags=0):
        self.net = net
        self.flags = flags
        self.h = nif_create(net, mesh, precision, seed, flags)

    def close(self):
        if self.h is not None:
            nif_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, tables, weights, s=None):
        nif_set_params(self.h, NIF_PARAM_TABLES, tables)
        for i, w in enumerate(weights):
            nif_set_params(self.h, NIF_PARAM_LAYER0 + i, w)
        if s is not None:
            nif_set_params(self.h, NIF_PARAM_LOGVAR, s)

    def get_params(self):
        net = self.net
        tables = nif_get_params(self.h, NIF_PARAM_TABLES).reshape(net.levels, 1 << net.log2_table, net.feats)
        ws = [nif_get_params(self.h, NIF_PARAM_LAYER0 + i).reshape(o, i_)
              for i, (o, i_) in enumerate(net.layer_shapes())]
        s = nif_get_params(self.h, NIF_PARAM_LOGVAR)
        return tables, ws, s

    def get_grads(self):
        net = self.net
        tables = nif_get_grad(self.h, NIF_PARAM_TABLES).reshape(net.levels, 1 << net.log2_table, net.feats)
        ws = [nif_get_grad(self.h, NIF_PARAM_LAYER0 + i).reshape(o, i_)
              for i, (o, i_) in enumerate(net.layer_shapes())]
        s = nif_get_grad(self.h, NIF_PARAM_LOGVAR)
        return tables, ws, s
