"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle.

This module only *generates inputs*: meshes, rays, deformation poses and
initial parameters. It holds none of the method's arithmetic (no deformation,
no traversal, no encoding, no network), so both sides of every parity test can
take their inputs from here without sharing code.

The paper's meshes (a cat and a dragon, Sec. 3.2 / Fig. 4) are not available;
the two shapes below stand in for them:

* a triangulated torus (R=0.35, r=0.15, 64x32 quads, 4096 triangles),
* a union of 16 seeded random ellipsoids (about 50k triangles),

both inside the unit cube, which is the rest space of the method (Sec. 2).
Every generator takes an explicit seed and uses numpy's PCG64, so the same
seed gives the same arrays on any machine.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

CENTER = np.array([0.5, 0.5, 0.5])

# Fixed seeds of the workloads: geometry, rays, poses, parameter init.
SEED_GEOMETRY = 1
SEED_RAYS = 2
SEED_POSES = 3
SEED_INIT = 4


@dataclass
class Mesh:
    verts: np.ndarray      # float32 [nv, 3], rest space, inside [0,1]^3
    tris: np.ndarray       # int32 [nt, 3], outward winding
    albedo: np.ndarray     # float32 [nt, 3] in [0,1]
    material: np.ndarray   # uint8 [nt]

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


def torus_mesh(R: float = 0.35, r: float = 0.15, n_major: int = 64,
               n_minor: int = 32) -> Mesh:
    """Torus about the z axis through the cube centre, 2*n_major*n_minor tris.

    Material of a triangle: floor(4*phi/(2*pi)) of the major angle phi of its
    centroid. Albedo: 0.5 + 0.4*sin(6*pi*c + {0, 2.1, 4.2}) per channel, c the
    sum of the centroid's coordinates.
    """
    phi = 2.0 * np.pi * np.arange(n_major) / n_major
    th = 2.0 * np.pi * np.arange(n_minor) / n_minor
    P, T = np.meshgrid(phi, th, indexing="ij")
    x = (R + r * np.cos(T)) * np.cos(P)
    y = (R + r * np.cos(T)) * np.sin(P)
    z = r * np.sin(T)
    verts = np.stack([x, y, z], -1).reshape(-1, 3) + CENTER
    tris = []
    for i in range(n_major):
        i1 = (i + 1) % n_major
        for j in range(n_minor):
            j1 = (j + 1) % n_minor
            a, b = i * n_minor + j, i1 * n_minor + j
            c, d = i1 * n_minor + j1, i * n_minor + j1
            # winding chosen so (b-a)x(c-a) points away from the tube axis
            tris.append((a, b, c))
            tris.append((a, c, d))
    tris = np.asarray(tris, dtype=np.int32)
    cen = verts[tris].mean(axis=1)
    phic = np.mod(np.arctan2(cen[:, 1] - 0.5, cen[:, 0] - 0.5), 2 * np.pi)
    material = np.minimum(np.floor(4 * phic / (2 * np.pi)), 3).astype(np.uint8)
    s = cen.sum(axis=1)
    albedo = 0.5 + 0.4 * np.sin(2 * np.pi * 3 * s[:, None] + np.array([0.0, 2.1, 4.2]))
    return Mesh(verts.astype(np.float32), tris, albedo.astype(np.float32), material)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a uniform unit quaternion (Shoemake 1992)."""
    u1, u2, u3 = rng.random(3)
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
                  math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3),
                  math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def ellipsoid_union_mesh(seed: int = SEED_GEOMETRY, n: int = 16, n_u: int = 69,
                         n_v: int = 69) -> Mesh:
    """Union of n seeded ellipsoids: centres U[0.3,0.7]^3, radii U[0.05,0.25].

    Each ellipsoid is a UV sphere with n_u segments and n_v stacks (pole fans),
    2*n_u*(n_v-1) triangles. Triangles whose three vertices all lie strictly
    inside another ellipsoid are dropped, which approximates the union's
    surface; with 69x69 the union keeps about 50k triangles. Material =
    ellipsoid index mod 4; albedo = a seeded colour per ellipsoid.
    """
    rng = np.random.default_rng(seed)
    cents = rng.uniform(0.3, 0.7, size=(n, 3))
    radii = rng.uniform(0.05, 0.25, size=(n, 3))
    rots = [_random_rotation(rng) for _ in range(n)]
    cols = rng.uniform(0.1, 0.9, size=(n, 3))
    # unit sphere UV mesh
    th = np.pi * np.arange(1, n_v) / n_v           # stacks (no poles)
    ph = 2 * np.pi * np.arange(n_u) / n_u
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    ring = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    sph = np.concatenate([ring, [[0, 0, 1.0]], [[0, 0, -1.0]]], 0)
    top, bot = len(ring), len(ring) + 1
    ft = []
    for j in range(n_u):
        j1 = (j + 1) % n_u
        ft.append((top, j, j1))                     # north fan (stack 0 near +z)
    for i in range(n_v - 2):
        for j in range(n_u):
            j1 = (j + 1) % n_u
            a, b = i * n_u + j, i * n_u + j1
            c, d = (i + 1) * n_u + j1, (i + 1) * n_u + j
            ft.append((a, d, c))
            ft.append((a, c, b))
    last = (n_v - 2) * n_u
    for j in range(n_u):
        j1 = (j + 1) % n_u
        ft.append((bot, last + j1, last + j))
    ft = np.asarray(ft, dtype=np.int64)
    # orient outward: check with the first triangle of the unit sphere
    a, b, c = sph[ft[n_u]]
    if np.dot(np.cross(b - a, c - a), (a + b + c) / 3) < 0:
        ft = ft[:, [0, 2, 1]]

    verts, tris, alb, mat = [], [], [], []
    base = 0
    for e in range(n):
        v = (sph * radii[e]) @ rots[e].T + cents[e]
        keep = np.ones(len(ft), bool)
        for o in range(n):
            if o == e:
                continue
            local = (v - cents[o]) @ rots[o] / radii[o]   # into o's unit sphere frame
            inside = (local * local).sum(1) < 1.0
            keep &= ~inside[ft].all(1)
        t = ft[keep] + base
        verts.append(v)
        tris.append(t)
        alb.append(np.repeat(cols[e][None], len(t), 0))
        mat.append(np.full(len(t), e % 4))
        base += len(v)
    return Mesh(np.concatenate(verts).astype(np.float32),
                np.concatenate(tris).astype(np.int32),
                np.concatenate(alb).astype(np.float32),
                np.concatenate(mat).astype(np.uint8))


def sphere_rays(n: int, seed: int = SEED_RAYS, radius: float = 2.0,
                center=CENTER) -> np.ndarray:
    """Rays [n, 8] float32 = (o.xyz, d.xyz, tmin, tmax).

    Origins uniform on the sphere of the given radius about the cube centre,
    each aimed at a point uniform in [0,1]^3; d has unit length; tmin = 0 and
    tmax = 1e30.
    """
    rng = np.random.default_rng(seed)
    z = rng.uniform(-1, 1, n)
    a = rng.uniform(0, 2 * np.pi, n)
    s = np.sqrt(1 - z * z)
    o = np.asarray(center) + radius * np.stack([s * np.cos(a), s * np.sin(a), z], -1)
    tgt = rng.uniform(0, 1, (n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    out = np.zeros((n, 8), np.float32)
    out[:, 0:3] = o
    out[:, 3:6] = d
    out[:, 6] = 0.0
    out[:, 7] = 1e30
    return out


def chained_segments(n: int, seed: int, voxel_res: int = 64, gap: float = 0.1,
                     margin: float = 0.01) -> tuple:
    """Linearized segments shaped like a training batch, without any method
    arithmetic: straight lines through the cube (origin uniform on the
    radius-2 sphere about the centre, aimed at a uniform point of the cube),
    each clipped to [-margin, 1+margin]^3 and cut at spacings U[0.2, 1.2]/N
    along the line; piece j runs from cut j to cut j+1, so a piece's entry
    point is the previous piece's exit point bit for bit (float32), except
    where a piece is left out (probability `gap`, like a ray crossing an
    empty voxel). Points up to `margin` outside the cube occur near the
    faces.

    Returns (lin [n, 8] float32 = p0.xyz, p1.xyz, l_def, l_rest with both
    lengths |p1 - p0|, voxel [n] uint32 = the voxel i + N(j + Nk) holding the
    piece's midpoint, clamped into the grid)."""
    rng = np.random.default_rng(seed)
    rows, vox = [], []
    total = 0
    lo, hi = -margin, 1.0 + margin
    while total < n:
        z = rng.uniform(-1, 1)
        a = rng.uniform(0, 2 * np.pi)
        r = math.sqrt(1 - z * z)
        o = CENTER + 2.0 * np.array([r * math.cos(a), r * math.sin(a), z])
        d = rng.uniform(0, 1, 3) - o
        d /= np.linalg.norm(d)
        with np.errstate(divide="ignore"):
            t1 = (lo - o) / d
            t2 = (hi - o) / d
        ta = np.max(np.minimum(t1, t2))
        tb = np.min(np.maximum(t1, t2))
        if not tb > ta:
            continue
        cuts = [ta]
        while True:
            c = cuts[-1] + rng.uniform(0.2, 1.2) / voxel_res
            if c >= tb:
                break
            cuts.append(c)
        cuts.append(tb)
        pts = (o[None, :] + np.asarray(cuts)[:, None] * d[None, :]).astype(np.float32)
        keep = rng.random(len(pts) - 1) >= gap
        for j in np.nonzero(keep)[0]:
            p0, p1 = pts[j], pts[j + 1]
            ln = np.float32(np.linalg.norm(p1.astype(np.float64) - p0.astype(np.float64)))
            rows.append(np.concatenate([p0, p1, [ln, ln]]).astype(np.float32))
            mid = np.clip(np.floor(0.5 * (p0.astype(np.float64) + p1) * voxel_res), 0, voxel_res - 1).astype(np.int64)
            vox.append(mid[0] + voxel_res * (mid[1] + voxel_res * mid[2]))
        total = len(rows)
    return np.stack(rows[:n]), np.asarray(vox[:n], np.uint32)


def camera_rays(width: int = 1920, height: int = 1080, grid: int = 4, eye=(0.5, -0.65, 0.95),
                target=CENTER, vfov_deg: float = 48.0) -> tuple:
    """Primary rays of one frame of a grid x grid world of instances seen by
    one camera: the image is cut into grid x grid tiles and tile k shows
    instance k, whose rays are given in the instance's own frame (the rest
    cube [0,1]^3) from a pinhole at `eye` looking at `target` (z up).
    Returns (rays [width*height, 8] float32 grouped by instance, offsets
    [grid*grid + 1] int32)."""
    tw, th = width // grid, height // grid
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, [0.0, 0.0, 1.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    t = np.tan(np.radians(vfov_deg) / 2)
    ys, xs = np.meshgrid((np.arange(th) + 0.5) / th, (np.arange(tw) + 0.5) / tw, indexing="ij")
    sx = (2 * xs - 1) * t * tw / th
    sy = (1 - 2 * ys) * t
    d = fwd + sx[..., None] * right + sy[..., None] * up
    d = (d / np.linalg.norm(d, axis=-1, keepdims=True)).reshape(-1, 3)
    tile = np.zeros((tw * th, 8), np.float32)
    tile[:, 0:3] = eye
    tile[:, 3:6] = d
    tile[:, 7] = 1e30
    n_inst = grid * grid
    rays = np.concatenate([tile] * n_inst)
    offs = (np.arange(n_inst + 1) * tw * th).astype(np.int32)
    return rays, offs


def animated_poses(n_inst: int, n_frames: int = 120, amplitude: float = 1.0, seed: int = SEED_POSES):
    """Poses [n_frames, n_inst, 3]: parameter j of instance i at frame f is
    amplitude * sin(2 pi f / n_frames + phi_ij), phases seeded U[0, 2 pi)."""
    phi = np.random.default_rng(seed).uniform(0, 2 * np.pi, (n_inst, 3))
    f = np.arange(n_frames)[:, None, None]
    return (amplitude * np.sin(2 * np.pi * f / n_frames + phi[None])).astype(np.float32)


def poses(n: int, seed: int = SEED_POSES, kind: str = "all") -> np.ndarray:
    """Deformation parameters [n, 3] float32 = (bend, twist, taper).

    kind="twist": twist angle-rate U[-pi/2, pi/2], bend = taper = 0.
    kind="all": each parameter U[-1, 1].
    """
    rng = np.random.default_rng(seed)
    out = np.zeros((n, 3), np.float32)
    if kind == "twist":
        out[:, 1] = rng.uniform(-np.pi / 2, np.pi / 2, n)
    elif kind == "all":
        out[:] = rng.uniform(-1, 1, (n, 3))
    else:
        raise ValueError(kind)
    return out


@dataclass
class NetConfig:
    """Sizes of the encoding and network (symbols of the method, Eq. 1)."""
    voxel_res: int = 16        # N
    pe_bands: int = 4          # F
    levels: int = 8            # L
    feats: int = 2             # F_d
    log2_table: int = 14       # T = 2^t
    base_res: int = 4          # N_min
    growth: float = 1.5        # b
    mlp_depth: int = 2         # hidden layers H
    mlp_width: int = 32        # W
    n_materials: int = 4       # M
    encoding: str = "composed"  # Eq. 1 read as psi = phi o gamma ("composed") or [gamma, phi] ("concat")
    faces: str = "triangles"    # deformed voxel faces: two triangles each, or bilinear patches ("bilinear")

    @property
    def n_terms(self) -> int:            # P = 1 + 2F
        return 1 + 2 * self.pe_bands

    @property
    def point_width(self) -> int:        # features of one end point: P*L*F_d, or 3P + L*F_d concatenated
        if self.encoding == "concat":
            return 3 * self.n_terms + self.levels * self.feats
        return self.n_terms * self.levels * self.feats

    @property
    def in_dim(self) -> int:             # 2 end points, padded to 16 columns when concatenated
        if self.encoding == "concat":
            return (2 * self.point_width + 15) // 16 * 16
        return 2 * self.point_width

    @property
    def out_dim(self) -> int:            # occ, dist, normal(3), albedo(3), material(M)
        return 8 + self.n_materials

    @property
    def out_pad(self) -> int:            # output rows stored, padded to 16
        return max(16, ((self.out_dim + 15) // 16) * 16)

    def layer_shapes(self):
        """[(out, in)] of every weight matrix, input layer first."""
        dims = [self.in_dim] + [self.mlp_width] * self.mlp_depth
        shapes = [(dims[i + 1], dims[i]) for i in range(self.mlp_depth)]
        shapes.append((self.out_pad, self.mlp_width))
        return shapes

    def asdict(self):
        return asdict(self)


def init_params(cfg: NetConfig, seed: int = SEED_INIT):
    """Initial parameters: (tables, [weights], s).

    tables  float32 [L, T, F_d] ~ U[-1e-4, 1e-4]
    weights float32 [out, in] per layer, Kaiming-uniform U[-sqrt(6/in), sqrt(6/in)];
            the padding rows of the output layer (index >= out_dim) are zero.
    s       float32 [5] log-variances of the five tasks, zero.
    """
    rng = np.random.default_rng(seed)
    T = 1 << cfg.log2_table
    tables = rng.uniform(-1e-4, 1e-4, (cfg.levels, T, cfg.feats)).astype(np.float32)
    ws = []
    for (o, i) in cfg.layer_shapes():
        b = math.sqrt(6.0 / i)
        w = rng.uniform(-b, b, (o, i)).astype(np.float32)
        ws.append(w)
    ws[-1][cfg.out_dim:, :] = 0.0
    s = np.zeros(5, np.float32)
    return tables, ws, s


def zipf_ray_counts(n_inst: int = 64, s: float = 1.2, lo: int = 1024,
                    hi: int = 262144, total: int = 1 << 22,
                    seed: int = SEED_RAYS) -> np.ndarray:
    """Per-instance ray counts, Zipf(s) over ranks, clamped to [lo, hi].

    n_r = clamp(floor(C * r^-s), lo, hi) for rank r = 1..n_inst with C found by
    bisection so that the sum is as close as possible to `total`; ranks are
    permuted over the instances by the seed.
    """
    r = np.arange(1, n_inst + 1, dtype=np.float64)

    def counts(C):
        return np.clip(np.floor(C * r ** (-s)), lo, hi).astype(np.int64)

    a, b = 1.0, 1e12
    for _ in range(200):
        m = 0.5 * (a + b)
        if counts(m).sum() < total:
            a = m
        else:
            b = m
    c = counts(b)
    rng = np.random.default_rng(seed)
    return c[rng.permutation(n_inst)]


# ---------------------------------------------------------------------------
# Workloads (shapes and sizes of the five measured configurations)
# ---------------------------------------------------------------------------

WORKLOADS = {
    # plain FP32 forward: torus at 16^3, twist only, 4096 rays
    "torus16_fwd": dict(shape="torus", net=NetConfig(16, 4, 8, 2, 14, 4, 1.5, 2, 32, 4),
                        n_rays=4096, pose_kind="twist"),
    # FP32 train step: ellipsoid union at 64^3, 2^18 segments per step
    "ellipsoids64_train": dict(shape="ellipsoids", net=NetConfig(64, 4, 16, 2, 19, 4, 1.5, 3, 64, 4),
                               n_segments=1 << 18, pose_kind="all"),
    # precision: torus at 128^3, 2^22 rays, network of the torus16 workload
    "torus128_query": dict(shape="torus", net=NetConfig(128, 4, 8, 2, 14, 4, 1.5, 2, 32, 4),
                           n_rays=1 << 22, pose_kind="all"),
    # batching: 64 torus instances at 16^3, Zipf ray counts, L=16, T=2^19, 3x64
    "torus16x64_batch": dict(shape="torus", net=NetConfig(16, 4, 16, 2, 19, 4, 1.5, 3, 64, 4),
                             n_inst=64, pose_kind="all"),
    # animated frame loop: 16 ellipsoid-union instances at 256^3, T=2^21, MLP 4x64, BF16;
    # 1920x1080 primary + shadow rays per frame, 120 frames, pose fitting in the loop
    "ellipsoids256_frame": dict(shape="ellipsoids", net=NetConfig(256, 4, 16, 2, 21, 4, 1.5, 4, 64, 4),
                                n_inst=16, width=1920, height=1080, frames=120),
}


def make_mesh(shape: str) -> Mesh:
    if shape == "torus":
        return torus_mesh()
    if shape == "ellipsoids":
        return ellipsoid_union_mesh(SEED_GEOMETRY)
    raise ValueError(shape)
