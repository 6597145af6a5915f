"""FP64 CPU oracle of the voxel deformation-aware neural intersection function.

TEST INFRASTRUCTURE ONLY: only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this package. It shares no code with
the CUDA library (`paper_2604_24666_gb300/csrc`) and never imports it.

The oracle follows the paper step by step, in float64:

* geometry (C, `nif_oracle.c`): deformation and inverse (Sec. 2), voxelization
  (Sec. 2), ray / deformed-voxel segments (Sec. 2.1-2.2), linearized-segment
  labels (Sec. 2), exact deformed-space hits;
* the hybrid encoding psi = phi o gamma (Eq. 1, Sec. 2.3), its backward;
  and the other reading of Eq. 1, the concatenation psi = [gamma, phi];
* the MLP (Sec. 2, Fig. 2d) forward and backward, and the same with the
  16-bit storage points of the mixed-precision path rounded (Sec. 3);
* the task losses and the uncertainty weighting (Sec. 2.4);
* Adam;
* the segmented-ray distance and hit reconstruction (Sec. 2.2).

Where the paper is silent the oracle takes the readings that the library
states in its header (`include/nif.h`); every such reading is listed with the
design notes of the repository.

Integer decisions made from floating point (hash-grid cell indices) are taken
in float32, the precision the kernels use: the oracle rounds the grid
coordinate u to float32 and forms the float32 product u*N_l before the floor.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

K_BEND = 0.75          # bend curvature per unit bend parameter
EPS_DIST = 1e-2        # epsilon of the log-space distance loss (voxel units)
TASKS = ("distance", "normal", "albedo", "material", "occlusion")


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (FP64, no FMA contraction)."""
    src = os.path.join(_HERE, "nif_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp, fp, ip, lp = (np.ctypeslib.ndpointer(np.float64, flags="C"),
                              np.ctypeslib.ndpointer(np.float32, flags="C"),
                              np.ctypeslib.ndpointer(np.int32, flags="C"),
                              np.ctypeslib.ndpointer(np.int64, flags="C"))
            u8 = np.ctypeslib.ndpointer(np.uint8, flags="C")
            L.or_deform.argtypes = [dp, dp, dp, ctypes.c_long]
            L.or_inverse.argtypes = [dp, dp, dp, ctypes.c_long]
            L.or_jacobians.argtypes = [dp, dp, dp, dp, ctypes.c_long]
            L.or_voxelize.argtypes = [ctypes.c_int, fp, ip, ctypes.c_int, u8, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_long]
            L.or_voxelize.restype = ctypes.c_long
            L.or_segments.argtypes = [ctypes.c_int, u8, dp, fp, ctypes.c_long, ctypes.c_int, ip, ip,
                                      dp, dp, dp, ctypes.c_int, ctypes.c_void_p]
            L.or_bilinear_hits.argtypes = [dp, dp, dp, dp, dp, dp, dp, dp, dp]
            L.or_bilinear_hits.restype = ctypes.c_int
            L.or_segments.restype = ctypes.c_long
            L.or_labels.argtypes = [lp, ip, fp, ip, fp, u8, ctypes.c_long, ip, dp, dp, u8, dp, dp, dp,
                                    u8, dp]
            L.or_exact_hits.argtypes = [dp, ip, ctypes.c_int, fp, ctypes.c_long, dp, ip]
            L.or_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().or_num_threads())


# ---------------------------------------------------------------------------
# Deformation (Sec. 2; family and parameterisation are our reading)
# ---------------------------------------------------------------------------

def _pose(pose) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(pose, np.float64).reshape(3))


def deform(pose, x) -> np.ndarray:
    """D(x): rest -> deformed, D = Bend o Twist o Taper about the cube centre."""
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 3))
    y = np.empty_like(x)
    lib().or_deform(_pose(pose), x, y, len(x))
    return y


def inverse(pose, y) -> np.ndarray:
    """D^-1(y): deformed -> rest (closed form)."""
    y = np.ascontiguousarray(np.asarray(y, np.float64).reshape(-1, 3))
    x = np.empty_like(y)
    lib().or_inverse(_pose(pose), y, x, len(y))
    return x


def jacobians(pose, x):
    """(J, Jp): dD/dx [n,3,3] and dD/d(bend,twist,taper) [n,3,3] at rest points x."""
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 3))
    J = np.empty((len(x), 9))
    Jp = np.empty((len(x), 9))
    lib().or_jacobians(_pose(pose), x, J, Jp, len(x))
    return J.reshape(-1, 3, 3), Jp.reshape(-1, 3, 3)


# ---------------------------------------------------------------------------
# Voxelization (Sec. 2)
# ---------------------------------------------------------------------------

def voxelize(N: int, mesh):
    """(occ [N^3] uint8 x-fastest, tri_ptr [N^3+1] int64, tri_idx int32)."""
    verts = np.ascontiguousarray(mesh.verts, np.float32)
    tris = np.ascontiguousarray(mesh.tris, np.int32)
    occ = np.zeros(N ** 3, np.uint8)
    total = lib().or_voxelize(N, verts, tris, len(tris), occ, None, None, 0)
    ptr = np.zeros(N ** 3 + 1, np.int64)
    idx = np.zeros(max(total, 1), np.int32)
    lib().or_voxelize(N, verts, tris, len(tris), occ, ptr.ctypes.data, idx.ctypes.data, total)
    return occ, ptr, idx[:total]


# ---------------------------------------------------------------------------
# Segments (Sec. 2.1, Sec. 2.2)
# ---------------------------------------------------------------------------

class Segments:
    """Ragged segment lists: ray r owns rows [off[r], off[r+1])."""

    def __init__(self, count, vox, t0, t1, margin):
        self.count = count
        self.off = np.concatenate([[0], np.cumsum(count)]).astype(np.int64)
        self.vox = vox
        self.t0 = t0
        self.t1 = t1
        self.margin = margin
        self.ray = np.repeat(np.arange(len(count)), count)

    def __len__(self):
        return int(self.off[-1])


def bilinear_hits(o, d, P00, P10, P01, P11):
    """Hits of the line o + t d with the bilinear patch of the four corners
    (u along P00 -> P10, v along P00 -> P01): list of (t, u, v), and the
    distance between the two hit points when there are two (else inf)."""
    f = lambda a: np.ascontiguousarray(a, np.float64).reshape(3)
    t = np.zeros(2)
    uv = np.zeros(4)
    sep = np.zeros(1)
    n = lib().or_bilinear_hits(f(o), f(d), f(P00), f(P10), f(P01), f(P11), t, uv, sep)
    return [(t[i], uv[2 * i], uv[2 * i + 1]) for i in range(n)], (sep[0] if n == 2 else np.inf)


def segments(N: int, occ, pose, rays, max_per_ray: int = 512, faces: str = "triangles", field=None) -> Segments:
    """Ray / deformed voxel segments (Sec. 2.1, 2.2). faces: "triangles" (each
    face split along the diagonal from its lowest lattice corner) or
    "bilinear" (each face the bilinear patch of its four corners). With a
    learned deformation field (`field`, see `deform_field`) the hull corners
    are D(lattice corners) of the composed deformation."""
    assert faces in ("triangles", "bilinear")
    lattice = None
    if field is not None:
        g = np.arange(N + 1, dtype=np.float64) / N
        Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
        lattice = np.ascontiguousarray(deform_field(pose, field, np.stack([X, Y, Z], -1).reshape(-1, 3)))
    rays = np.ascontiguousarray(rays, np.float32)
    n = len(rays)
    cnt = np.zeros(n, np.int32)
    vox = np.zeros(n * max_per_ray, np.int32)
    t0 = np.zeros(n * max_per_ray)
    t1 = np.zeros(n * max_per_ray)
    mar = np.zeros(n)
    ov = lib().or_segments(N, np.ascontiguousarray(occ, np.uint8), _pose(pose), rays, n,
                           max_per_ray, cnt, vox, t0, t1, mar, int(faces == "bilinear"),
                           None if lattice is None else lattice.ctypes.data_as(ctypes.c_void_p))
    if ov:
        raise RuntimeError(f"{ov} rays exceed {max_per_ray} segments")
    sel = (np.arange(max_per_ray)[None, :] < cnt[:, None]).reshape(-1)
    return Segments(cnt, vox[sel], t0[sel], t1[sel], mar)


def linearize(pose, rays, seg: Segments, field=None):
    """Rest-space straight segment of every (ray, voxel) segment (Sec. 2).

    x0 = o + t0 d, x1 = o + t1 d in deformed space; p0 = D^-1(x0), p1 = D^-1(x1)
    (with `field`, the inverse of the composed deformation, `inverse_field`).
    Returns p0, p1 [S,3], l_def = |x1 - x0|, l_rest = |p1 - p0|.
    """
    rays = np.asarray(rays, np.float64)
    o = rays[seg.ray, 0:3]
    d = rays[seg.ray, 3:6]
    x0 = o + seg.t0[:, None] * d
    x1 = o + seg.t1[:, None] * d
    inv = (lambda y: inverse_field(pose, field, y)) if field is not None else (lambda y: inverse(pose, y))
    p0 = inv(x0)
    p1 = inv(x1)
    return p0, p1, np.linalg.norm(x1 - x0, axis=1), np.linalg.norm(p1 - p0, axis=1)


def labels(mesh, tri_ptr, tri_idx, vox, p0, p1):
    """Ground truth of the linearized rest segments: dict of arrays (Sec. 2)."""
    n = len(vox)
    out = dict(occ=np.zeros(n, np.uint8), tpar=np.zeros(n), normal=np.zeros((n, 3)),
               albedo=np.zeros((n, 3)), material=np.zeros(n, np.uint8), margin=np.zeros(n))
    lib().or_labels(np.ascontiguousarray(tri_ptr, np.int64), np.ascontiguousarray(tri_idx, np.int32),
                    np.ascontiguousarray(mesh.verts, np.float32), np.ascontiguousarray(mesh.tris, np.int32),
                    np.ascontiguousarray(mesh.albedo, np.float32), np.ascontiguousarray(mesh.material, np.uint8),
                    n, np.ascontiguousarray(vox, np.int32), np.ascontiguousarray(p0, np.float64),
                    np.ascontiguousarray(p1, np.float64), out["occ"], out["tpar"], out["normal"],
                    out["albedo"], out["material"], out["margin"])
    return out


def exact_hits(mesh, pose, rays):
    """First hit of each ray with the deformed mesh (vertices mapped by D)."""
    dv = np.ascontiguousarray(deform(pose, mesh.verts.astype(np.float64)))
    rays = np.ascontiguousarray(rays, np.float32)
    t = np.zeros(len(rays))
    tri = np.zeros(len(rays), np.int32)
    lib().or_exact_hits(dv, np.ascontiguousarray(mesh.tris, np.int32), len(mesh.tris), rays,
                        len(rays), t, tri)
    return t, tri


# ---------------------------------------------------------------------------
# Hybrid encoding psi = phi o gamma (Eq. 1)
# ---------------------------------------------------------------------------

def level_res(cfg):
    """N_l = floor(N_min * b^l), l = 0..L-1."""
    return [int(np.floor(cfg.base_res * cfg.growth ** l)) for l in range(cfg.levels)]


def level_dense(cfg):
    T = 1 << cfg.log2_table
    return [(n + 1) ** 3 <= T for n in level_res(cfg)]


def gamma(cfg, p):
    """gamma(x) = [x, sin(2^k x), cos(2^k x)]_{k<F} as P = 1+2F 3-vectors [n, P, 3]
    and their grid coordinates u in [0,1]^3 (x as is, (g+1)/2 for sin/cos)."""
    p = np.clip(np.asarray(p, np.float64), 0.0, 1.0)
    g = [p]
    for k in range(cfg.pe_bands):
        g.append(np.sin((2.0 ** k) * p))
        g.append(np.cos((2.0 ** k) * p))
    g = np.stack(g, 1)
    u = g.copy()
    u[:, 1:] = 0.5 * (g[:, 1:] + 1.0)
    return g, u


def grid_index(cfg, l, corner):
    """Table row of integer grid vertex corner [.., 3] (uint32 arithmetic)."""
    Nl = level_res(cfg)[l]
    T = 1 << cfg.log2_table
    c = corner.astype(np.uint64)
    if (Nl + 1) ** 3 <= T:
        return (c[..., 0] + c[..., 1] * (Nl + 1) + c[..., 2] * (Nl + 1) ** 2).astype(np.int64)
    h = (c[..., 0] * np.uint64(1)) ^ ((c[..., 1] * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)) \
        ^ ((c[..., 2] * np.uint64(805459861)) & np.uint64(0xFFFFFFFF))
    return (h & np.uint64(T - 1)).astype(np.int64)


def _cell(cfg, l, u):
    """Cell of u at level l: float32 decision q = fl32(fl32(u) * N_l), i0, w."""
    Nl = level_res(cfg)[l]
    uf = np.asarray(u, np.float32).astype(np.float64)
    q = (uf * Nl).astype(np.float32).astype(np.float64)
    i0 = np.minimum(np.floor(q), Nl - 1).astype(np.int64)
    w = q - i0
    return i0, w


_CORNERS = np.array([[(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], np.int64)


def grid_encode(cfg, tables, u):
    """phi(u) for points u [n, 3]: [n, L, F_d], trilinear per level (Eq. 1)."""
    tables = np.asarray(tables, np.float64)
    out = np.zeros((len(u), cfg.levels, cfg.feats))
    for l in range(cfg.levels):
        i0, w = _cell(cfg, l, u)
        for c in _CORNERS:
            idx = grid_index(cfg, l, i0 + c)
            wt = np.prod(np.where(c == 1, w, 1.0 - w), axis=1)
            out[:, l, :] += wt[:, None] * tables[l][idx]
    return out


def encode_points(cfg, tables, p):
    """psi(p) = phi(gamma(p)) for rest points p [n,3]: [n, P*L*F_d],
    ordered [term][level][feature]."""
    _, u = gamma(cfg, p)
    n, P = u.shape[0], u.shape[1]
    feats = np.stack([grid_encode(cfg, tables, u[:, t]) for t in range(P)], 1)
    return feats.reshape(n, -1)


def encode_points_concat(cfg, tables, p):
    """The concatenation reading of Eq. 1: psi(p) = [gamma(p), phi(p)] for rest
    points p [n,3]: [n, 3P + L*F_d]. gamma as its raw values ordered
    [term][coordinate] (x, then sin(2^k x), cos(2^k x) for k < F), phi the
    grid at u = p (clamped to [0,1]^3), ordered [level][feature]."""
    g, u = gamma(cfg, p)
    n = g.shape[0]
    return np.concatenate([g.reshape(n, -1), grid_encode(cfg, tables, u[:, 0]).reshape(n, -1)], 1)


def encode_segments(cfg, tables, p0, p1):
    """MLP input of a segment: psi(p0) (+) psi(p1), [S, 2*P*L*F_d]; with the
    concatenation reading the two [S, 3P + L*F_d] halves, zero-padded to
    cfg.in_dim columns."""
    if getattr(cfg, "encoding", "composed") == "concat":
        x = np.concatenate([encode_points_concat(cfg, tables, p0), encode_points_concat(cfg, tables, p1)], 1)
        return np.pad(x, ((0, 0), (0, cfg.in_dim - x.shape[1])))
    return np.concatenate([encode_points(cfg, tables, p0), encode_points(cfg, tables, p1)], 1)


def encode_points_backward(cfg, tables, p, dfeat):
    """Gradients of sum(dfeat * psi(p)): (dtables [L,T,F_d], dp [n,3])."""
    tables = np.asarray(tables, np.float64)
    res = level_res(cfg)
    pc = np.asarray(p, np.float64)
    inside = (pc >= 0.0) & (pc <= 1.0)
    pcl = np.clip(pc, 0.0, 1.0)
    g, u = gamma(cfg, pc)
    n, P = u.shape[0], u.shape[1]
    dfeat = np.asarray(dfeat, np.float64).reshape(n, P, cfg.levels, cfg.feats)
    dtab = np.zeros_like(tables)
    du = np.zeros((n, P, 3))
    for t in range(P):
        for l in range(cfg.levels):
            i0, w = _cell(cfg, l, u[:, t])
            gl = dfeat[:, t, l, :]
            for c in _CORNERS:
                idx = grid_index(cfg, l, i0 + c)
                f = np.where(c == 1, w, 1.0 - w)
                wt = np.prod(f, axis=1)
                np.add.at(dtab[l], idx, wt[:, None] * gl)
                val = (tables[l][idx] * gl).sum(1)
                for a in range(3):
                    others = np.prod(np.delete(f, a, axis=1), axis=1)
                    sgn = 1.0 if c[a] == 1 else -1.0
                    du[:, t, a] += sgn * others * res[l] * val
    # chain through u(gamma(p)): x-term du/dp = 1; sin term 0.5*2^k cos(2^k p); cos term -0.5*2^k sin(2^k p)
    dp = du[:, 0, :].copy()
    for k in range(cfg.pe_bands):
        f = 2.0 ** k
        dp += du[:, 1 + 2 * k, :] * 0.5 * f * np.cos(f * pcl)
        dp += du[:, 2 + 2 * k, :] * (-0.5) * f * np.sin(f * pcl)
    dp = np.where(inside, dp, 0.0)
    return dtab, dp


def encode_points_concat_backward(cfg, tables, p, dfeat):
    """Gradients of sum(dfeat * [gamma(p), phi(p)]) (dfeat [n, 3P + L*F_d]):
    (dtables [L,T,F_d], dp [n,3]). The table gradient comes from the phi part
    only; dp adds d gamma/dp (1 for x, 2^k cos(2^k p) for sin, -2^k sin(2^k p)
    for cos, per coordinate) and d phi/dp (the trilinear weights'
    derivatives times N_l), zero where p was clamped."""
    tables = np.asarray(tables, np.float64)
    res = level_res(cfg)
    pc = np.asarray(p, np.float64)
    inside = (pc >= 0.0) & (pc <= 1.0)
    pcl = np.clip(pc, 0.0, 1.0)
    n, P = len(pc), cfg.n_terms
    dfeat = np.asarray(dfeat, np.float64)
    dg = dfeat[:, :3 * P].reshape(n, P, 3)
    dphi = dfeat[:, 3 * P:3 * P + cfg.levels * cfg.feats].reshape(n, cfg.levels, cfg.feats)
    dp = dg[:, 0, :].copy()
    for k in range(cfg.pe_bands):
        f = 2.0 ** k
        dp += dg[:, 1 + 2 * k, :] * f * np.cos(f * pcl)
        dp -= dg[:, 2 + 2 * k, :] * f * np.sin(f * pcl)
    dtab = np.zeros_like(tables)
    for l in range(cfg.levels):
        i0, w = _cell(cfg, l, pcl)
        gl = dphi[:, l, :]
        for c in _CORNERS:
            idx = grid_index(cfg, l, i0 + c)
            fw = np.where(c == 1, w, 1.0 - w)
            np.add.at(dtab[l], idx, np.prod(fw, axis=1)[:, None] * gl)
            val = (tables[l][idx] * gl).sum(1)
            for a in range(3):
                sgn = 1.0 if c[a] == 1 else -1.0
                dp[:, a] += sgn * np.prod(np.delete(fw, a, axis=1), axis=1) * res[l] * val
    return dtab, np.where(inside, dp, 0.0)


# ---------------------------------------------------------------------------
# MLP (Sec. 2, Fig. 2d): ReLU hidden layers, no bias, linear output
# ---------------------------------------------------------------------------

def mlp_forward(ws, x):
    """Returns (out [S, O], acts) with acts[i] the input of layer i."""
    acts = [np.asarray(x, np.float64)]
    h = acts[0]
    for i, w in enumerate(ws):
        z = h @ np.asarray(w, np.float64).T
        if i < len(ws) - 1:
            h = np.maximum(z, 0.0)
            acts.append(h)
        else:
            h = z
    return h, acts


def mlp_backward(ws, acts, dout):
    """(dws, dx) for dL/dout."""
    g = np.asarray(dout, np.float64)
    dws = [None] * len(ws)
    for i in range(len(ws) - 1, -1, -1):
        w = np.asarray(ws[i], np.float64)
        dws[i] = g.T @ acts[i]
        g = g @ w
        if i > 0:
            g = g * (acts[i] > 0)
    return dws, g


def mlp_forward_rounded(ws, x, rnd):
    """MLP forward of the mixed-precision path (Sec. 3 trains with 16-bit
    operands): inputs, weights and the stored hidden activations pass through
    `rnd` (rounding to the 16-bit type, given by the caller); products and
    sums are exact (float64). Returns (out, acts) like mlp_forward, acts being
    the rounded inputs of each layer."""
    h = rnd(np.asarray(x, np.float64))
    acts = [h]
    for i, w in enumerate(ws):
        z = h @ rnd(np.asarray(w, np.float64)).T
        if i < len(ws) - 1:
            h = rnd(np.maximum(z, 0.0))
            acts.append(h)
        else:
            h = z
    return h, acts


def mlp_backward_rounded(ws, acts, dout, scale, rnd):
    """Backward of the mixed-precision path for the loss multiplied by
    `scale` (loss scaling): the output gradient and each layer's gradient are
    rounded by `rnd` where the path stores them in 16 bits, i.e.
    dY_H = rnd(scale * dout), dY_l = rnd((dY_{l+1} W_{l+1}) * [act > 0]),
    weights rounded as in the forward. Returns (dws, dx), both multiplied by
    `scale` (dx = dY_0 W_0 unrounded)."""
    g = rnd(scale * np.asarray(dout, np.float64))
    dws = [None] * len(ws)
    for i in range(len(ws) - 1, -1, -1):
        w = rnd(np.asarray(ws[i], np.float64))
        dws[i] = g.T @ acts[i]
        g = g @ w
        if i > 0:
            g = rnd(g * (acts[i] > 0))
    return dws, g


# ---------------------------------------------------------------------------
# Losses (Sec. 2.4)
# ---------------------------------------------------------------------------

def _sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def _softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


FLAG_FIXED_TASK_WEIGHTS = 1
FLAG_SIGMOID_DISTANCE = 2
SQRT3 = float(np.sqrt(3.0))


def loss(cfg, out, lab, s, l_rest, flags=0):
    """Uncertainty-weighted multi-task loss and its gradients.

    out   [S, O] network outputs: 0 occupancy logit, 1 distance (ReLU),
          2:5 normal, 5:8 albedo logits (sigmoid), 8:8+M material logits.
    lab   dict of occ, tpar, normal, albedo, material (from `labels`).
    s     [5] log-variances (distance, normal, albedo, material, occlusion).
    l_rest [S] rest-segment lengths; the distance target is the rest hit
          distance in voxel units, tpar * l_rest * N.
    flags (ablation, the "Deformed" baseline): FLAG_FIXED_TASK_WEIGHTS holds
    s at 0 (total = sum 0.5 L_reg + L_cls, ds = 0); FLAG_SIGMOID_DISTANCE uses
    the head sqrt(3) sigmoid(z) with a plain squared error.
    Returns (total, parts [5], dout [S, O], ds [5]).
    """
    out = np.asarray(out, np.float64)
    s = np.asarray(s, np.float64)
    S = out.shape[0]
    M = cfg.n_materials
    hit = lab["occ"].astype(bool)
    nh = int(hit.sum())
    dout = np.zeros_like(out)
    parts = np.zeros(5)
    fixed = bool(flags & FLAG_FIXED_TASK_WEIGHTS)
    if fixed:
        s = np.zeros(5)
    es = np.exp(-s)
    if nh > 0:
        zh = out[hit]
        y = lab["tpar"][hit] * np.asarray(l_rest)[hit] * cfg.voxel_res
        if flags & FLAG_SIGMOID_DISTANCE:
            sg = _sigmoid(zh[:, 1])
            e = SQRT3 * sg - y
            parts[0] = (e * e).sum() / nh
            gd = 0.5 * es[0] * 2.0 * e * SQRT3 * sg * (1 - sg) / nh
        else:
            # distance: ReLU head, MSE of logs
            dh = np.maximum(zh[:, 1], 0.0)
            e = np.log(dh + EPS_DIST) - np.log(y + EPS_DIST)
            parts[0] = (e * e).sum() / nh
            gd = 0.5 * es[0] * 2.0 * e / (dh + EPS_DIST) / nh * (zh[:, 1] > 0)
        # normal: 1 - cosine
        nhat = zh[:, 2:5]
        n = lab["normal"][hit]
        nn = np.maximum(np.linalg.norm(nhat, axis=1), 1e-8)
        dot = (nhat * n).sum(1)
        parts[1] = (1.0 - dot / nn).sum() / nh
        gn = -(n / nn[:, None] - (dot / nn ** 3)[:, None] * nhat) * (0.5 * es[1] / nh)
        # albedo: sigmoid + L1
        ah = _sigmoid(zh[:, 5:8])
        diff = ah - lab["albedo"][hit]
        parts[2] = np.abs(diff).sum() / (3 * nh)
        ga = np.sign(diff) * ah * (1 - ah) * (0.5 * es[2] / (3 * nh))
        # material: cross entropy
        zm = zh[:, 8:8 + M]
        mx = zm.max(1, keepdims=True)
        lse = mx[:, 0] + np.log(np.exp(zm - mx).sum(1))
        m = lab["material"][hit].astype(np.int64)
        parts[3] = (lse - zm[np.arange(nh), m]).sum() / nh
        sm = np.exp(zm - lse[:, None])
        sm[np.arange(nh), m] -= 1.0
        gm = sm * (es[3] / nh)
        g = np.zeros((nh, out.shape[1]))
        g[:, 1] = gd
        g[:, 2:5] = gn
        g[:, 5:8] = ga
        g[:, 8:8 + M] = gm
        dout[hit] = g
    # occlusion: BCE with logits over all segments
    z0 = out[:, 0]
    occ = lab["occ"].astype(np.float64)
    parts[4] = (_softplus(z0) - occ * z0).sum() / S
    dout[:, 0] = (_sigmoid(z0) - occ) * (es[4] / S)
    wreg = np.array([0.5, 0.5, 0.5, 1.0, 1.0])
    if fixed:
        return float((wreg * parts).sum()), parts, dout, np.zeros(5)
    total = float((wreg * es * parts + 0.5 * s).sum())
    ds = -wreg * es * parts + 0.5
    return total, parts, dout, ds


# ---------------------------------------------------------------------------
# Adam
# ---------------------------------------------------------------------------

def adam(theta, m, v, g, step, lr, b1=0.9, b2=0.99, eps=1e-15):
    """One Adam step (1-based step); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
# Reconstruction along the segmented ray (Sec. 2.2)
# ---------------------------------------------------------------------------

def reconstruct(cfg, pose, rays, seg: Segments, out, p0, p1, l_def, l_rest, flags=0, field=None):
    """Per ray: first segment k (in list order) with sigmoid(occ) > 0.5;
    D = sum_{j<k} (delta_j + l_j) + delta_k + t_k with t_k the predicted rest
    distance mapped to deformed length, t_k = (dist/N) * l_def/l_rest, clamped
    to [0, l_def]. The normal is J_D^{-T} n_rest normalised, evaluated at the
    predicted rest hit point. Returns dict hit, D, normal, albedo, material, k.
    """
    rays = np.asarray(rays, np.float64)
    n = len(rays)
    res = dict(hit=np.zeros(n, np.uint8), D=np.full(n, np.inf), normal=np.zeros((n, 3)),
               albedo=np.zeros((n, 3)), material=np.zeros(n, np.uint8), k=np.full(n, -1))
    for r in range(n):
        a, b = seg.off[r], seg.off[r + 1]
        prev = rays[r, 0:3]
        acc = 0.0
        for j in range(a, b):
            x0 = rays[r, 0:3] + seg.t0[j] * rays[r, 3:6]
            x1 = rays[r, 0:3] + seg.t1[j] * rays[r, 3:6]
            delta = np.linalg.norm(x0 - prev)
            if out[j, 0] > 0.0:
                dvox = SQRT3 * _sigmoid(out[j, 1]) if flags & FLAG_SIGMOID_DISTANCE else max(out[j, 1], 0.0)
                trest = dvox / cfg.voxel_res
                tk = trest * l_def[j] / l_rest[j] if l_rest[j] > 0 else 0.0
                tk = min(max(tk, 0.0), l_def[j])
                res["hit"][r] = 1
                res["k"][r] = j - a
                res["D"][r] = acc + delta + tk
                frac = trest / l_rest[j] if l_rest[j] > 0 else 0.0
                ph = p0[j] + frac * (p1[j] - p0[j])
                J = jacobian_field(pose, field, ph[None])[0] if field is not None else jacobians(pose, ph[None])[0][0]
                nd = np.linalg.solve(J.T, out[j, 2:5])
                res["normal"][r] = nd / max(np.linalg.norm(nd), 1e-30)
                res["albedo"][r] = _sigmoid(out[j, 5:8])
                res["material"][r] = int(np.argmax(out[j, 8:8 + cfg.n_materials]))
                break
            acc += delta + np.linalg.norm(x1 - x0)
            prev = x1
    return res


# ---------------------------------------------------------------------------
# Gradient with respect to the deformation parameters (pose fitting)
# ---------------------------------------------------------------------------

def pose_gradient(cfg, tables, pose, p0, p1, dfeat, field=None):
    """d/d(bend, twist, taper) of sum(dfeat * [psi(p0) (+) psi(p1)]) where the
    rest points are p = D^-1(x; pose) of fixed deformed points x.

    By the implicit function theorem, D(p(theta); theta) = x gives
    dp/dtheta = -J_D(p)^-1 dD/dtheta(p); the encoding's input gradient comes
    from `encode_points_backward`. With a learned field (D = D_theta o (I+u))
    the pose acts at q = p + u(p): dp/dtheta = -(I + du/dp)^-1
    J_theta(q)^-1 dD_theta/dtheta(q).
    """
    concat = getattr(cfg, "encoding", "composed") == "concat"
    half = cfg.point_width if concat else dfeat.shape[1] // 2
    back = encode_points_concat_backward if concat else encode_points_backward
    g = np.zeros(3)
    for p, df in ((p0, dfeat[:, :half]), (p1, dfeat[:, half:2 * half])):
        _, dp = back(cfg, tables, p, df)
        q = p if field is None else p + field_displacement(field, p)
        J, Jp = jacobians(pose, q)
        dpdth = -np.linalg.solve(J, Jp)            # [n, 3, 3]: d q_i / d theta_j
        if field is not None:
            dpdth = np.linalg.solve(np.eye(3)[None] + field_grad(field, p), dpdth)
        g += np.einsum("ni,nij->j", dp, dpdth)
    return g


# ---------------------------------------------------------------------------
# Learned deformation field (the paper's Sec. 4 names learning deformation
# fields jointly with intersection prediction as future work and defines no
# field; this is our reading)
# ---------------------------------------------------------------------------
#
# A field is an array delta [G, G, G, 3] (index [k, j, i] = node
# (i, j, k)/(G-1) of a lattice over the rest cube, G >= 2) of rest-space
# displacements, interpolated trilinearly: u(p) = sum_n w_n(p) delta_n with
# p clamped to [0,1]^3 first. The deformation of an instance with pose theta
# and field delta is the composition
#     D(p) = D_theta(p + u(p)),
# the field acting in rest space before the parameterised deformation, so
# that a zero field is the analytic deformation and a zero pose the field
# alone. Voxel hulls are the hexahedra of D(lattice corners) as for the
# analytic deformation. Its inverse takes q = D_theta^-1(x) (closed form)
# and solves F(p) = p + u(p) - q = 0. While the Lipschitz bound l of u
# (`field_lipschitz`) is below 1, p -> q - u(p) is a contraction, so the
# root is unique, and |p - p*| <= |F(p)| / (1 - l) for any p.


def field_cell(field, p):
    """Cell, weights and clamping of rest points p [n,3] in the field's
    lattice: (i0 [n,3] int, t [n,3] in [0,1], inside [n,3] bool)."""
    G = field.shape[0]
    p = np.asarray(p, np.float64)
    inside = (p >= 0.0) & (p <= 1.0)
    s = np.clip(p, 0.0, 1.0) * (G - 1)
    i0 = np.minimum(np.floor(s), G - 2).astype(np.int64)
    return i0, s - i0, inside


def field_displacement(field, p):
    """u(p) [n,3]: trilinear interpolation of the node displacements."""
    field = np.asarray(field, np.float64)
    i0, t, _ = field_cell(field, p)
    u = np.zeros((len(i0), 3))
    for c in _CORNERS:
        w = np.prod(np.where(c == 1, t, 1.0 - t), axis=1)
        n = i0 + c
        u += w[:, None] * field[n[:, 2], n[:, 1], n[:, 0]]
    return u


def field_grad(field, p):
    """du/dp [n,3,3] (row: component of u, column: coordinate of p); zero
    along a coordinate where p lies outside [0,1] (u is constant there)."""
    field = np.asarray(field, np.float64)
    G = field.shape[0]
    i0, t, inside = field_cell(field, p)
    g = np.zeros((len(i0), 3, 3))
    for c in _CORNERS:
        n = i0 + c
        d = field[n[:, 2], n[:, 1], n[:, 0]]
        f = np.where(c == 1, t, 1.0 - t)
        for a in range(3):
            others = np.prod(np.delete(f, a, axis=1), axis=1)
            sgn = 1.0 if c[a] == 1 else -1.0
            g[:, :, a] += (sgn * (G - 1) * others)[:, None] * d
    return g * inside[:, None, :]


def deform_field(pose, field, p):
    """D(p) = D_theta(p + u(p))."""
    p = np.asarray(p, np.float64).reshape(-1, 3)
    return deform(pose, p + field_displacement(field, p))


def jacobian_field(pose, field, p):
    """dD/dp [n,3,3] = J_theta(p + u(p)) (I + du/dp)."""
    p = np.asarray(p, np.float64).reshape(-1, 3)
    J, _ = jacobians(pose, p + field_displacement(field, p))
    return np.einsum("nij,njk->nik", J, np.eye(3)[None] + field_grad(field, p))


def field_lipschitz(field):
    """Bound l on the spectral norm of du/dp over the cube: within a cell,
    du/dp_a is a convex combination of the cell's four edge differences
    along a times (G-1), so ||du/dp||_2 <= ||du/dp||_F <= the root of the
    sum over a of (G-1)^2 max_edge |delta_b - delta_a|^2."""
    f = np.asarray(field, np.float64)
    G = f.shape[0]
    m = np.zeros((G - 1, G - 1, G - 1, 3))
    # axis 0 of the array is z (k), 1 is y (j), 2 is x (i)
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        e = np.linalg.norm(np.diff(f, axis=ax), axis=-1) * (G - 1)     # edges along this axis
        # the four edges of a cell along this axis: max over the other two axes' two positions
        others = [o for o in (0, 1, 2) if o != ax]
        for o in others:
            e = np.maximum(np.take(e, range(0, e.shape[o] - 1), axis=o), np.take(e, range(1, e.shape[o]), axis=o))
        m[..., a] = e
    return float(np.sqrt((m ** 2).sum(-1)).max())


def field_inverse(field, q, tol=1e-14, max_iter=100):
    """p with p + u(p) = q, by Newton's method on F(p) = p + u(p) - q from
    p = q - u(q); the field must satisfy field_lipschitz < 1."""
    q = np.asarray(q, np.float64).reshape(-1, 3)
    p = q - field_displacement(field, q)
    for _ in range(max_iter):
        F = p + field_displacement(field, p) - q
        if np.abs(F).max() <= tol:
            break
        J = np.eye(3)[None] + field_grad(field, p)
        p = p - np.linalg.solve(J, F[..., None])[..., 0]
    return p


def inverse_field(pose, field, x):
    """D^-1(x) of the composed deformation: Newton on the field after the
    closed-form inverse of the pose."""
    return field_inverse(field, inverse(pose, x))


def field_from_pose(G, pose):
    """Field whose nodes carry the analytic deformation: delta_n =
    D_theta(x_n) - x_n, so that the field alone (zero pose) agrees with the
    pose at every node and between nodes up to the trilinear interpolation
    error."""
    g = np.arange(G, dtype=np.float64) / (G - 1)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    x = np.stack([X, Y, Z], -1).reshape(-1, 3)
    return (deform(pose, x) - x).reshape(G, G, G, 3)


def field_gradient(cfg, tables, pose, field, p0, p1, dfeat):
    """d/d(delta) [G,G,G,3] of sum(dfeat * [psi(p0) (+) psi(p1)]) where the
    rest points are p = D^-1(x) of fixed deformed points x. With q =
    D_theta^-1(x) fixed, p + u(p) = q gives dp/d(delta_n) = -(I + du/dp)^-1
    w_n(p), so the gradient is -sum over points of w_n(p) (I + du/dp)^-T dL/dp
    with dL/dp from `encode_points_backward`."""
    concat = getattr(cfg, "encoding", "composed") == "concat"
    half = cfg.point_width if concat else dfeat.shape[1] // 2
    back = encode_points_concat_backward if concat else encode_points_backward
    field = np.asarray(field, np.float64)
    out = np.zeros_like(field)
    for p, df in ((p0, dfeat[:, :half]), (p1, dfeat[:, half:2 * half])):
        _, dp = back(cfg, tables, p, df)
        A = np.eye(3)[None] + field_grad(field, p)
        v = np.linalg.solve(np.transpose(A, (0, 2, 1)), dp[..., None])[..., 0]     # (I + du/dp)^-T dL/dp
        i0, t, _ = field_cell(field, p)
        for c in _CORNERS:
            w = np.prod(np.where(c == 1, t, 1.0 - t), axis=1)
            n = i0 + c
            np.add.at(out, (n[:, 2], n[:, 1], n[:, 0]), -w[:, None] * v)
    return out
