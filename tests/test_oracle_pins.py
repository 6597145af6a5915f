"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against a closed form, an invariant, an
independent textbook algorithm (Amanatides-Woo grid traversal, polygon
clipping, an analytic quartic) or central finite differences, so that a
plausible mistake in the oracle (a dropped term, a sign, a swapped index)
fails at least one of them. None of these tests needs a GPU.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_24666_gb300 import synth as S

C = np.array([0.5, 0.5, 0.5])


# ---------------------------------------------------------------------------
# Deformation (bend o twist o taper)
# ---------------------------------------------------------------------------

def _barr_bend(k, p):
    """Textbook Barr bend with R = 1/k: X = R - (R-x) cos(kz), Z = (R-x) sin(kz)."""
    R = 1.0 / k
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    return np.stack([R - (R - x) * np.cos(k * z), y, (R - x) * np.sin(k * z)], 1)


def _twist(th, p):
    a = th * p[:, 2]
    return np.stack([np.cos(a) * p[:, 0] - np.sin(a) * p[:, 1],
                     np.sin(a) * p[:, 0] + np.cos(a) * p[:, 1], p[:, 2]], 1)


def _taper(ka, p):
    s = 1 + ka * p[:, 2]
    return np.stack([s * p[:, 0], s * p[:, 1], p[:, 2]], 1)


def test_deform_identity_pose():
    x = np.random.default_rng(0).uniform(0, 1, (1000, 3))
    assert np.array_equal(O.deform((0, 0, 0), x), x)
    assert np.array_equal(O.inverse((0, 0, 0), x), x)


@pytest.mark.parametrize("pose", [(0.5, 0, 0), (-1, 0, 0), (0, 1.2, 0), (0, 0, -0.8),
                                  (0.9, -1.0, 0.6), (-0.4, 1.5, -1.0)])
def test_deform_matches_textbook_composition(pose):
    """D = c + Bend(Twist(Taper(x - c))) with Barr's bend written with R = 1/k."""
    x = np.random.default_rng(1).uniform(0, 1, (2000, 3))
    p = _taper(pose[2], x - C)
    p = _twist(pose[1], p)
    if pose[0] != 0:
        p = _barr_bend(O.K_BEND * pose[0], p)
    np.testing.assert_allclose(O.deform(pose, x), p + C, atol=1e-13, rtol=0)


def test_deform_roundtrip_random_poses():
    rng = np.random.default_rng(2)
    worst = 0.0
    for _ in range(200):
        pose = rng.uniform(-1, 1, 3) * np.array([1, math.pi / 2, 1])
        x = rng.uniform(0, 1, (500, 3))
        y = O.deform(pose, x)
        worst = max(worst, np.abs(O.inverse(pose, y) - x).max())
        yb = rng.uniform(0.1, 0.9, (100, 3))
        worst = max(worst, np.abs(O.deform(pose, O.inverse(pose, yb)) - yb).max())
    assert worst < 1e-13


def test_bend_small_curvature_is_continuous():
    """The bend tends to the identity with error ~ k z^2 / 2 as k -> 0."""
    x = np.random.default_rng(3).uniform(0, 1, (100, 3))
    for b in (1e-3, 1e-6, 1e-9, 0.0):
        y = O.deform((b, 0, 0), x)
        bound = O.K_BEND * abs(b) * 0.25 + 1e-15
        assert np.abs(y - x).max() <= bound
    # first-order term: dX/dk = z^2/2 at x = c + (0, 0, z)
    z = 0.4
    p = np.array([[0.5, 0.5, 0.5 + z]])
    y = O.deform((1e-4, 0, 0), p)
    np.testing.assert_allclose((y[0, 0] - 0.5) / (O.K_BEND * 1e-4), z * z / 2, rtol=1e-4)


def test_twist_rotates_horizontal_slices():
    """A point at height z turns by theta * (z - 0.5) about the vertical axis."""
    th = 1.3
    r, phi, z = 0.3, 0.7, 0.8
    x = np.array([[0.5 + r * math.cos(phi), 0.5 + r * math.sin(phi), z]])
    y = O.deform((0, th, 0), x)[0]
    a = phi + th * (z - 0.5)
    np.testing.assert_allclose(y, [0.5 + r * math.cos(a), 0.5 + r * math.sin(a), z], atol=1e-15)


def test_jacobians_match_finite_differences():
    rng = np.random.default_rng(4)
    h = 1e-6
    for _ in range(20):
        pose = rng.uniform(-1, 1, 3)
        x = rng.uniform(0, 1, (5, 3))
        J, Jp = O.jacobians(pose, x)
        for a in range(3):
            e = np.zeros(3); e[a] = h
            fd = (O.deform(pose, x + e) - O.deform(pose, x - e)) / (2 * h)
            np.testing.assert_allclose(J[:, :, a], fd, atol=1e-8)
            fdp = (O.deform(pose + e, x) - O.deform(pose - e, x)) / (2 * h)
            np.testing.assert_allclose(Jp[:, :, a], fdp, atol=1e-8)
    # at zero bend (the series branch)
    x = rng.uniform(0, 1, (5, 3))
    _, Jp = O.jacobians((0.0, 0.3, 0.2), x)
    e = np.array([h, 0, 0])
    fd = (O.deform((h, 0.3, 0.2), x) - O.deform((-h, 0.3, 0.2), x)) / (2 * h)
    np.testing.assert_allclose(Jp[:, :, 0], fd, atol=1e-8)


# ---------------------------------------------------------------------------
# Voxelization against polygon clipping
# ---------------------------------------------------------------------------

def _clip_overlap(tri, lo, hi):
    """Sutherland-Hodgman: clip the triangle by the six half-spaces of the box."""
    poly = [np.asarray(v, np.float64) for v in tri]
    for a in range(3):
        for side, bound in ((1, lo[a]), (-1, hi[a])):
            out = []
            for i in range(len(poly)):
                P, Q = poly[i], poly[(i + 1) % len(poly)]
                fp, fq = side * (P[a] - bound), side * (Q[a] - bound)
                if fp >= 0:
                    out.append(P)
                if (fp >= 0) != (fq >= 0):
                    t = fp / (fp - fq)
                    out.append(P + t * (Q - P))
            poly = out
            if not poly:
                return False
    return True


def test_voxelize_matches_clipping():
    rng = np.random.default_rng(5)
    N = 6
    for trial in range(40):
        c = rng.uniform(0.1, 0.9, 3)
        v = (c + rng.normal(0, 0.15, (3, 3))).clip(0.001, 0.999).astype(np.float32)
        mesh = S.Mesh(v, np.array([[0, 1, 2]], np.int32), np.zeros((1, 3), np.float32),
                      np.zeros(1, np.uint8))
        occ, ptr, idx = O.voxelize(N, mesh)
        eps = 1e-7
        ref = np.zeros(N ** 3, np.uint8)
        for k in range(N):
            for j in range(N):
                for i in range(N):
                    lo = np.array([i, j, k]) / N - eps
                    hi = (np.array([i, j, k]) + 1) / N + eps
                    ref[i + N * (j + N * k)] = _clip_overlap(v.astype(np.float64), lo, hi)
        assert np.array_equal(occ, ref), trial
        assert np.array_equal(np.diff(ptr), occ.astype(np.int64))


def test_voxelize_covers_surface_samples():
    mesh = S.torus_mesh()
    N = 16
    occ, ptr, idx = O.voxelize(N, mesh)
    rng = np.random.default_rng(6)
    P = mesh.verts[mesh.tris].astype(np.float64)
    uv = rng.uniform(0, 1, (len(P), 8, 2))
    uv = np.where(uv.sum(-1, keepdims=True) > 1, 1 - uv, uv)
    pts = P[:, None, 0] + uv[..., :1] * (P[:, None, 1] - P[:, None, 0]) + uv[..., 1:] * (P[:, None, 2] - P[:, None, 0])
    ijk = np.clip(np.floor(pts * N).astype(int), 0, N - 1).reshape(-1, 3)
    assert occ[ijk[:, 0] + N * (ijk[:, 1] + N * ijk[:, 2])].all()
    # every listed triangle of a voxel has a sample or a vertex within the dilated voxel box
    assert occ.sum() == (np.diff(ptr) > 0).sum()


# ---------------------------------------------------------------------------
# Segments: identity pose against a textbook DDA; invariants under deformation
# ---------------------------------------------------------------------------

def _dda(o, d, N):
    """Amanatides-Woo traversal of the N^3 grid over [0,1]^3; [(voxel, t_in, t_out)]."""
    tin, tout = -np.inf, np.inf
    for a in range(3):
        if d[a] == 0:
            if not (0 <= o[a] <= 1):
                return []
            continue
        t0, t1 = (0 - o[a]) / d[a], (1 - o[a]) / d[a]
        tin, tout = max(tin, min(t0, t1)), min(tout, max(t0, t1))
    if tin >= tout or tout <= 0:
        return []
    tin = max(tin, 0.0)
    p = o + tin * d
    ijk = np.clip(np.floor(p * N).astype(int), 0, N - 1)
    step = np.sign(d).astype(int)
    tmax = np.array([((ijk[a] + (step[a] > 0)) / N - o[a]) / d[a] if d[a] != 0 else np.inf for a in range(3)])
    tdel = np.array([abs(1.0 / (N * d[a])) if d[a] != 0 else np.inf for a in range(3)])
    out = []
    t = tin
    while True:
        a = int(np.argmin(tmax))
        tn = min(tmax[a], tout)
        out.append((ijk[0] + N * (ijk[1] + N * ijk[2]), t, tn))
        if tmax[a] >= tout:
            break
        t = tmax[a]
        ijk[a] += step[a]
        tmax[a] += tdel[a]
        if not (0 <= ijk[a] < N):
            break
    return out


def test_segments_identity_pose_equal_dda():
    mesh = S.torus_mesh()
    N = 8
    occ, _, _ = O.voxelize(N, mesh)
    rays = S.sphere_rays(400, seed=11)
    seg = O.segments(N, occ, (0, 0, 0), rays)
    checked = 0
    for r in range(len(rays)):
        if seg.margin[r] < 1e-9:
            continue
        o, d = rays[r, :3].astype(np.float64), rays[r, 3:6].astype(np.float64)
        ref = [(v, a, b) for (v, a, b) in _dda(o, d, N) if occ[v] and b - a > 0]
        got = list(range(seg.off[r], seg.off[r + 1]))
        assert [v for v, _, _ in ref] == [int(seg.vox[j]) for j in got], r
        for (v, a, b), j in zip(ref, got):
            assert abs(a - seg.t0[j]) < 1e-12 and abs(b - seg.t1[j]) < 1e-12
        checked += len(got)
    assert checked > 500


@pytest.mark.parametrize("pose", [(0.8, -0.9, 0.5), (-1.0, 1.0, -1.0)])
def test_segments_deformed_invariants(pose):
    mesh = S.torus_mesh()
    N = 16
    occ, _, _ = O.voxelize(N, mesh)
    rays = S.sphere_rays(1500, seed=12)
    seg = O.segments(N, occ, pose, rays)
    # sorted by entry; exits never before entries
    assert np.all(seg.t1 > seg.t0)
    for r in range(len(rays)):
        a, b = seg.off[r], seg.off[r + 1]
        assert np.all(np.diff(seg.t0[a:b]) >= 0)
    # hulls of face-adjacent voxels share their face: consecutive segments touch or leave a gap
    gaps = [seg.t0[j + 1] - seg.t1[j] for r in range(len(rays)) for j in range(seg.off[r], seg.off[r + 1] - 1)]
    gaps = np.array(gaps)
    assert (gaps < -1e-9).mean() < 0.01
    assert (np.abs(gaps) < 1e-12).mean() > 0.5
    # every exact deformed-mesh hit lies inside a segment (up to the hull's flat faces)
    thit, tri = O.exact_hits(mesh, pose, rays)
    for r in np.nonzero(np.isfinite(thit))[0]:
        a, b = seg.off[r], seg.off[r + 1]
        inside = (seg.t0[a:b] - 2e-3 <= thit[r]) & (thit[r] <= seg.t1[a:b] + 2e-3)
        assert inside.any(), r


def _ray_torus(o, d, R=0.35, r=0.15):
    o = o - C
    G = o @ o + R * R - r * r
    B = o @ d
    c = [1.0, 4 * B, 4 * B * B + 2 * G - 4 * R * R * (d[0] ** 2 + d[1] ** 2),
         4 * B * G - 8 * R * R * (o[0] * d[0] + o[1] * d[1]), G * G - 4 * R * R * (o[0] ** 2 + o[1] ** 2)]
    roots = np.roots(c)
    ts = sorted(t.real for t in roots if abs(t.imag) < 1e-6 and t.real > 0)
    if not ts:
        return np.inf
    t = ts[0]
    for _ in range(5):  # Newton polish on the quartic
        f = np.polyval(c, t)
        df = np.polyval(np.polyder(c), t)
        if df != 0:
            t -= f / df
    return t


def test_exact_hits_match_analytic_torus():
    mesh = S.torus_mesh()
    rays = S.sphere_rays(600, seed=13)
    t, tri = O.exact_hits(mesh, (0, 0, 0), rays)
    sag = 0.15 * (1 - math.cos(math.pi / 32)) + 0.5 * (1 - math.cos(math.pi / 64))
    n_ok = 0
    for i in range(len(rays)):
        o, d = rays[i, :3].astype(np.float64), rays[i, 3:6].astype(np.float64)
        ta = _ray_torus(o, d)
        if not (np.isfinite(ta) and np.isfinite(t[i])):
            continue
        p = o + ta * d - C
        rho = math.hypot(p[0], p[1])
        n = np.array([p[0] * (1 - 0.35 / rho), p[1] * (1 - 0.35 / rho), p[2]])
        cosi = abs(n @ d) / np.linalg.norm(n)
        if cosi < 0.3:
            continue
        assert abs(t[i] - ta) <= sag / cosi + 1e-9, i
        n_ok += 1
    assert n_ok > 100


# ---------------------------------------------------------------------------
# Labels
# ---------------------------------------------------------------------------

def test_labels_identity_pose_give_exact_first_hit():
    """At the identity pose the linearized segment is the ray itself, so the
    first labelled segment reproduces the brute-force first hit exactly."""
    mesh = S.torus_mesh()
    N = 16
    occ, ptr, idx = O.voxelize(N, mesh)
    rays = S.sphere_rays(800, seed=14)
    pose = (0, 0, 0)
    seg = O.segments(N, occ, pose, rays)
    p0, p1, ld, lr = O.linearize(pose, rays, seg)
    lab = O.labels(mesh, ptr, idx, seg.vox, p0, p1)
    thit, tri = O.exact_hits(mesh, pose, rays)
    n = 0
    for r in range(len(rays)):
        a, b = seg.off[r], seg.off[r + 1]
        hits = np.nonzero(lab["occ"][a:b])[0]
        if seg.margin[r] < 1e-9 or (len(hits) and lab["margin"][a + hits[0]] < 1e-9):
            continue
        if not len(hits):
            assert not np.isfinite(thit[r])
            continue
        j = a + hits[0]
        D = seg.t0[j] + lab["tpar"][j] * (seg.t1[j] - seg.t0[j])
        assert abs(D - thit[r]) < 1e-9
        v0, v1, v2 = mesh.verts[mesh.tris[tri[r]]].astype(np.float64)
        nrm = np.cross(v1 - v0, v2 - v0)
        np.testing.assert_allclose(lab["normal"][j], nrm / np.linalg.norm(nrm), atol=1e-12)
        assert lab["material"][j] == mesh.material[tri[r]]
        n += 1
    assert n > 300


def test_label_distance_error_is_linearization_small():
    """Under deformation the GT-label distance (no network) differs from the
    exact deformed hit only by the local linearization, O(h^2)."""
    mesh = S.torus_mesh()
    N = 16
    occ, ptr, idx = O.voxelize(N, mesh)
    rays = S.sphere_rays(600, seed=15)
    pose = (0.7, -1.0, 0.5)
    seg = O.segments(N, occ, pose, rays)
    p0, p1, ld, lr = O.linearize(pose, rays, seg)
    lab = O.labels(mesh, ptr, idx, seg.vox, p0, p1)
    thit, _ = O.exact_hits(mesh, pose, rays)
    errs = []
    for r in range(len(rays)):
        a, b = seg.off[r], seg.off[r + 1]
        hits = np.nonzero(lab["occ"][a:b])[0]
        if len(hits) and np.isfinite(thit[r]):
            j = a + hits[0]
            D = seg.t0[j] + lab["tpar"][j] * ld[j]
            errs.append(abs(D - thit[r]))
    errs = np.array(errs)
    assert len(errs) > 200
    assert np.median(errs) < 2e-3 and (errs < 1e-2).mean() > 0.97


# ---------------------------------------------------------------------------
# Encoding (Eq. 1)
# ---------------------------------------------------------------------------

def test_level_resolutions():
    cfg = S.NetConfig(levels=16, log2_table=19)
    assert O.level_res(cfg) == [4, 6, 9, 13, 20, 30, 45, 68, 102, 153, 230, 345, 518, 778, 1167, 1751]
    assert O.level_dense(cfg) == [True] * 8 + [False] * 8
    assert O.level_dense(S.NetConfig(levels=8, log2_table=14)) == [True] * 5 + [False] * 3


def test_hash_of_axis_points():
    """With primes (1, 2654435761, 805459861) the hash of (i,0,0) is i, of
    (0,1,0) the second prime and of (0,0,1) the third, modulo T."""
    cfg = S.NetConfig(levels=16, log2_table=19)
    T = 1 << 19
    l = 15
    c = np.array([[7, 0, 0], [0, 1, 0], [0, 0, 1], [3, 1, 0]])
    got = O.grid_index(cfg, l, c)
    assert list(got) == [7, 2654435761 % T, 805459861 % T, (3 ^ 2654435761) % T]


def test_dense_levels_interpolate_linear_functions_exactly():
    cfg = S.NetConfig(levels=5, log2_table=14, feats=2)
    rng = np.random.default_rng(7)
    T = 1 << cfg.log2_table
    tables = np.zeros((cfg.levels, T, 2))
    coef = rng.normal(size=(cfg.levels, 2, 4))
    for l, Nl in enumerate(O.level_res(cfg)):
        g = np.arange(Nl + 1)
        I, J, K = np.meshgrid(g, g, g, indexing="ij")
        for f in range(2):
            vals = coef[l, f, 0] * I + coef[l, f, 1] * J + coef[l, f, 2] * K + coef[l, f, 3]
            tables[l, :(Nl + 1) ** 3, f] = vals.reshape(-1, order="F")   # x fastest
    u = rng.uniform(0, 1, (500, 3)).astype(np.float32).astype(np.float64)
    got = O.grid_encode(cfg, tables, u)
    for l, Nl in enumerate(O.level_res(cfg)):
        q = (u * Nl).astype(np.float32).astype(np.float64)
        for f in range(2):
            ref = q @ coef[l, f, :3] + coef[l, f, 3]
            np.testing.assert_allclose(got[:, l, f], ref, atol=1e-10)


def test_encoding_is_continuous_across_cells():
    cfg = S.NetConfig(levels=8, log2_table=10)
    tables = np.random.default_rng(8).uniform(-1, 1, (8, 1024, 2))
    rng = np.random.default_rng(9)
    p = rng.uniform(0.05, 0.95, (300, 3))
    d = rng.normal(size=(300, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    a = O.encode_points(cfg, tables, p)
    b = O.encode_points(cfg, tables, p + 1e-7 * d)
    # Lipschitz bound: 8 corners * max|table| * N_max * 2^F scale * step, generous
    assert np.abs(a - b).max() < 8 * 68 * 8 * 1e-7 * 4


def test_gamma_terms_closed_form():
    cfg = S.NetConfig(pe_bands=3)
    p = np.array([[0.0, 0.5, 1.0]])
    g, u = O.gamma(cfg, p)
    assert g.shape == (1, 7, 3)
    np.testing.assert_allclose(g[0, 0], [0, 0.5, 1.0])
    for k in range(3):
        np.testing.assert_allclose(g[0, 1 + 2 * k], np.sin(2.0 ** k * p[0]))
        np.testing.assert_allclose(g[0, 2 + 2 * k], np.cos(2.0 ** k * p[0]))
    np.testing.assert_allclose(u[0, 1], 0.5 * (np.sin(p[0]) + 1))
    # a constant table encodes to the constant on every term and level
    tables = np.full((cfg.levels, 1 << cfg.log2_table, 2), 0.25)
    np.testing.assert_allclose(O.encode_points(cfg, tables, p), 0.25, atol=1e-15)


def _tiny_cfg():
    return S.NetConfig(voxel_res=8, pe_bands=1, levels=3, feats=2, log2_table=6, base_res=2,
                       growth=1.5, mlp_depth=2, mlp_width=8, n_materials=4)


def test_encoding_backward_matches_finite_differences():
    cfg = _tiny_cfg()
    rng = np.random.default_rng(10)
    T = 1 << cfg.log2_table
    tables = rng.uniform(-1, 1, (cfg.levels, T, 2))
    p = rng.uniform(0.05, 0.95, (6, 3))
    w = rng.normal(size=(6, cfg.n_terms * cfg.levels * 2))
    dtab, dp = O.encode_points_backward(cfg, tables, p, w)
    f = lambda tb, pp: (O.encode_points(cfg, tb, pp) * w).sum()
    # tables: the encoding is linear in the table, so FD is exact up to rounding
    h = 1e-6
    for (l, i, c) in [(0, 3, 0), (1, 10, 1), (2, 17, 0), (2, 40, 1)]:
        e = np.zeros_like(tables); e[l, i, c] = h
        fd = (f(tables + e, p) - f(tables - e, p)) / (2 * h)
        assert abs(fd - dtab[l, i, c]) < 1e-7
    # points: piecewise smooth in p; the cell coordinate is rounded to float32
    # (about 6e-8), so the step must be large against that and small against a cell
    hp = 1e-4
    for a in range(3):
        e = np.zeros_like(p); e[:, a] = hp
        for s in range(len(p)):
            e1 = np.zeros_like(p); e1[s, a] = hp
            fd = (f(tables, p + e1) - f(tables, p - e1)) / (2 * hp)
            assert abs(fd - dp[s, a]) < 2e-3 * max(1, abs(dp[s, a])), (s, a)


# The concatenation reading of Eq. 1, psi = [gamma, phi]
def _tiny_concat_cfg():
    return S.NetConfig(voxel_res=8, pe_bands=2, levels=3, feats=2, log2_table=6, base_res=2,
                       growth=1.5, mlp_depth=2, mlp_width=8, n_materials=4, encoding="concat")


def test_concat_gamma_bands_and_layout():
    """gamma's raw values are pinned by identities between consecutive bands
    (sin 2a = 2 sin a cos a, cos 2a = 1 - 2 sin^2 a), sin^2 + cos^2 = 1, and
    a Taylor series for band 0; phi is the composed reading's x-term block;
    the segment row is [psi(p0), psi(p1), zeros]."""
    cfg = _tiny_concat_cfg()
    rng = np.random.default_rng(20)
    T = 1 << cfg.log2_table
    tables = rng.uniform(-1, 1, (cfg.levels, T, 2))
    p = rng.uniform(-0.1, 1.1, (50, 3))
    p[0] = [1e-3, 2e-3, 0.5]
    x = O.encode_points_concat(cfg, tables, p)
    P = cfg.n_terms
    assert x.shape == (50, 3 * P + cfg.levels * 2) and cfg.point_width == x.shape[1]
    g = x[:, :3 * P].reshape(50, P, 3)
    pc = np.clip(p, 0, 1)
    np.testing.assert_array_equal(g[:, 0], pc)
    for k in range(cfg.pe_bands):
        s, c = g[:, 1 + 2 * k], g[:, 2 + 2 * k]
        np.testing.assert_allclose(s * s + c * c, 1.0, atol=1e-14)
        if k + 1 < cfg.pe_bands:
            np.testing.assert_allclose(g[:, 3 + 2 * k], 2 * s * c, atol=1e-14)
            np.testing.assert_allclose(g[:, 4 + 2 * k], 1 - 2 * s * s, atol=1e-14)
    a = pc[0, :2]
    np.testing.assert_allclose(g[0, 1, :2], a - a ** 3 / 6 + a ** 5 / 120, rtol=1e-12)
    composed = S.NetConfig(**{**cfg.asdict(), "encoding": "composed"})
    np.testing.assert_array_equal(x[:, 3 * P:], O.encode_points(composed, tables, p)[:, :cfg.levels * 2])
    q = rng.uniform(0, 1, (50, 3))
    row = O.encode_segments(cfg, tables, p, q)
    w = cfg.point_width
    assert row.shape == (50, cfg.in_dim) and cfg.in_dim % 16 == 0 and cfg.in_dim >= 2 * w
    np.testing.assert_array_equal(row[:, :w], x)
    np.testing.assert_array_equal(row[:, w:2 * w], O.encode_points_concat(cfg, tables, q))
    assert not row[:, 2 * w:].any()


def test_concat_backward_matches_finite_differences():
    cfg = _tiny_concat_cfg()
    rng = np.random.default_rng(21)
    T = 1 << cfg.log2_table
    tables = rng.uniform(-1, 1, (cfg.levels, T, 2))
    p = rng.uniform(0.05, 0.95, (6, 3))
    p[5] = [1.02, 0.43, -0.01]                      # clamped x and z: zero gradient there (y off every cell face)
    w = rng.normal(size=(6, cfg.point_width))
    dtab, dp = O.encode_points_concat_backward(cfg, tables, p, w)
    f = lambda tb, pp: (O.encode_points_concat(cfg, tb, pp) * w).sum()
    h = 1e-6
    for (l, i, c) in [(0, 3, 0), (1, 10, 1), (2, 17, 0), (2, 40, 1)]:
        e = np.zeros_like(tables); e[l, i, c] = h
        fd = (f(tables + e, p) - f(tables - e, p)) / (2 * h)
        assert abs(fd - dtab[l, i, c]) < 1e-7
    hp = 1e-4
    for s in range(len(p)):
        for a in range(3):
            e1 = np.zeros_like(p); e1[s, a] = hp
            fd = (f(tables, p + e1) - f(tables, p - e1)) / (2 * hp)
            assert abs(fd - dp[s, a]) < 2e-3 * max(1, abs(dp[s, a])), (s, a, fd, dp[s, a])
    assert dp[5, 0] == 0 and dp[5, 2] == 0


def test_concat_pose_gradient_matches_finite_differences():
    cfg = _tiny_concat_cfg()
    rng = np.random.default_rng(22)
    T = 1 << cfg.log2_table
    tables = rng.uniform(-1, 1, (cfg.levels, T, 2))
    pose = np.array([0.4, -0.7, 0.5])
    x0 = rng.uniform(0.2, 0.8, (8, 3))
    x1 = x0 + rng.normal(0, 0.02, (8, 3))
    w = rng.normal(size=(8, cfg.in_dim))

    def f(th):
        return (O.encode_segments(cfg, tables, O.inverse(th, x0), O.inverse(th, x1)) * w).sum()

    g = O.pose_gradient(cfg, tables, pose, O.inverse(pose, x0), O.inverse(pose, x1), w)
    h = 1e-3
    for j in range(3):
        e = np.zeros(3); e[j] = h
        fd = (f(pose + e) - f(pose - e)) / (2 * h)
        assert abs(fd - g[j]) <= 5e-3 * max(1.0, abs(fd)), (j, fd, g[j])


# ---------------------------------------------------------------------------
# MLP, losses, Adam
# ---------------------------------------------------------------------------

def test_mlp_identity_weights():
    x = np.abs(np.random.default_rng(11).normal(size=(5, 4)))
    ws = [np.eye(4), np.eye(4), np.eye(4)]
    out, acts = O.mlp_forward(ws, x)
    np.testing.assert_allclose(out, x)
    out, _ = O.mlp_forward([np.eye(4), -np.eye(4)], x)
    np.testing.assert_allclose(out, -x)
    out, _ = O.mlp_forward([-np.eye(4), np.eye(4)], x)   # ReLU clamps
    np.testing.assert_allclose(out, 0 * x)


def _rand_labels(rng, n, M=4):
    occ = (rng.random(n) < 0.6).astype(np.uint8)
    nr = rng.normal(size=(n, 3)); nr /= np.linalg.norm(nr, axis=1, keepdims=True)
    return dict(occ=occ, tpar=rng.uniform(0.05, 1, n), normal=nr, albedo=rng.uniform(0, 1, (n, 3)),
                material=rng.integers(0, M, n).astype(np.uint8))


@pytest.mark.parametrize("flags", [0, O.FLAG_FIXED_TASK_WEIGHTS | O.FLAG_SIGMOID_DISTANCE])
def test_loss_and_mlp_gradients_match_finite_differences(flags):
    cfg = _tiny_cfg()
    rng = np.random.default_rng(12)
    n = 12
    ws = [rng.normal(size=sh) * 0.5 for sh in [(8, 10), (8, 8), (16, 8)]]
    x = rng.normal(size=(n, 10))
    lab = _rand_labels(rng, n)
    s = rng.normal(size=5) * 0.3
    lrest = rng.uniform(0.5, 1.0, n) / cfg.voxel_res

    def total(ws_, x_, s_):
        out, _ = O.mlp_forward(ws_, x_)
        return O.loss(cfg, out, lab, s_, lrest, flags)[0]

    out, acts = O.mlp_forward(ws, x)
    tot, parts, dout, ds = O.loss(cfg, out, lab, s, lrest, flags)
    dws, dx = O.mlp_backward(ws, acts, dout)
    h = 1e-6
    for li in range(3):
        for _ in range(6):
            i, j = rng.integers(0, ws[li].shape[0]), rng.integers(0, ws[li].shape[1])
            wp = [w.copy() for w in ws]; wm = [w.copy() for w in ws]
            wp[li][i, j] += h; wm[li][i, j] -= h
            fd = (total(wp, x, s) - total(wm, x, s)) / (2 * h)
            assert abs(fd - dws[li][i, j]) <= 1e-6 * max(1, abs(fd)), (li, i, j)
    for _ in range(10):
        i, j = rng.integers(0, n), rng.integers(0, 10)
        xp = x.copy(); xm = x.copy(); xp[i, j] += h; xm[i, j] -= h
        fd = (total(ws, xp, s) - total(ws, xm, s)) / (2 * h)
        assert abs(fd - dx[i, j]) <= 1e-6 * max(1, abs(fd))
    for t in range(5):
        e = np.zeros(5); e[t] = h
        fd = (total(ws, x, s + e) - total(ws, x, s - e)) / (2 * h)
        assert abs(fd - ds[t]) <= 1e-7


def test_loss_closed_forms():
    cfg = _tiny_cfg()
    rng = np.random.default_rng(13)
    n = 50
    lab = _rand_labels(rng, n)
    lab["occ"][:] = 1
    lrest = np.full(n, 1.0 / cfg.voxel_res)
    out = np.zeros((n, 16))
    y = lab["tpar"] * lrest * cfg.voxel_res
    out[:, 1] = y                                  # exact distance
    out[:, 2:5] = 3.0 * lab["normal"]               # parallel normal, any length
    a = np.clip(lab["albedo"], 1e-3, 1 - 1e-3)
    lab["albedo"] = a
    out[:, 5:8] = np.log(a / (1 - a))              # exact albedo
    out[np.arange(n), 8 + lab["material"].astype(int)] = 40.0   # confident class
    out[:, 0] = 40.0
    _, parts, _, _ = O.loss(cfg, out, lab, np.zeros(5), lrest)
    np.testing.assert_allclose(parts[:3], 0, atol=1e-12)
    assert parts[3] < 1e-15 and parts[4] < 1e-15
    # uncertainty weighting: ds = 0 at s = log(L) (regression), log(2L) (classification)
    out[:, 1] = 2 * y
    out[:, 0] = 0.0
    _, parts, _, _ = O.loss(cfg, out, lab, np.zeros(5), lrest)
    s_star = np.zeros(5)
    s_star[0] = np.log(parts[0])
    s_star[4] = np.log(2 * parts[4])
    _, _, _, ds = O.loss(cfg, out, lab, s_star, lrest)
    assert abs(ds[0]) < 1e-12 and abs(ds[4]) < 1e-12
    # occlusion loss of a zero logit is log 2
    np.testing.assert_allclose(parts[4], math.log(2))


def test_ablation_loss_closed_forms():
    """Fixed task weights: total = 0.5 (L_d + L_n + L_a) + L_m + L_o and no
    gradient for s; sigmoid distance head: exact when sqrt(3) sigmoid(z) = y."""
    cfg = _tiny_cfg()
    rng = np.random.default_rng(21)
    n = 40
    lab = _rand_labels(rng, n)
    lrest = np.full(n, 1.0 / cfg.voxel_res)
    out = rng.normal(size=(n, 16))
    s = rng.normal(size=5)
    tot, parts, _, ds = O.loss(cfg, out, lab, s, lrest, O.FLAG_FIXED_TASK_WEIGHTS)
    np.testing.assert_allclose(tot, 0.5 * parts[:3].sum() + parts[3:].sum())
    assert not ds.any()
    lab["occ"][:] = 1
    y = lab["tpar"] * lrest * cfg.voxel_res             # in [0, 1] < sqrt(3)
    q = y / np.sqrt(3.0)
    out[:, 1] = np.log(q / (1 - q))
    _, parts, _, _ = O.loss(cfg, out, lab, s, lrest, O.FLAG_SIGMOID_DISTANCE)
    assert parts[0] < 1e-20


def test_adam_first_step_is_signed_lr():
    g = np.array([1e-3, -2.0, 5.0])
    th, m, v = O.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-9)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.01 * g * g)


# ---------------------------------------------------------------------------
# Reconstruction along the segmented ray (Sec. 2.2)
# ---------------------------------------------------------------------------

def test_reconstruction_collinear_identity_and_normal():
    """For a straight ray with unit d, sum_{j<k}(delta_j + l_j) + delta_k = t0(k),
    and at the identity pose the reconstructed normal is the predicted one."""
    cfg = S.NetConfig()
    mesh = S.torus_mesh()
    occ, _, _ = O.voxelize(16, mesh)
    rays = S.sphere_rays(300, seed=16)
    rays[:, 3:6] /= np.linalg.norm(rays[:, 3:6].astype(np.float64), axis=1, keepdims=True).astype(np.float32)
    for pose in [(0, 0, 0), (0.5, 0.8, -0.6)]:
        seg = O.segments(16, occ, pose, rays)
        p0, p1, ld, lr = O.linearize(pose, rays, seg)
        rng = np.random.default_rng(17)
        out = rng.normal(size=(len(seg), 16))
        res = O.reconstruct(cfg, pose, rays, seg, out, p0, p1, ld, lr)
        dn = np.linalg.norm(rays[:, 3:6].astype(np.float64), axis=1)
        for r in np.nonzero(res["hit"])[0]:
            j = seg.off[r] + res["k"][r]
            tk = np.clip(max(out[j, 1], 0) / 16 * ld[j] / lr[j], 0, ld[j])
            assert abs(res["D"][r] - (seg.t0[j] * dn[r] + tk)) < 1e-12
            if pose == (0, 0, 0):
                nn = out[j, 2:5] / np.linalg.norm(out[j, 2:5])
                np.testing.assert_allclose(res["normal"][r], nn, atol=1e-12)


def test_pose_gradient_matches_finite_differences():
    """Gradient of sum(w * psi(D^-1(x; theta))) over theta for fixed deformed
    points x, against central differences of the oracle's own forward."""
    cfg = _tiny_cfg()
    rng = np.random.default_rng(14)
    T = 1 << cfg.log2_table
    tables = rng.uniform(-1, 1, (cfg.levels, T, 2))
    pose = np.array([0.4, -0.7, 0.5])
    x0 = rng.uniform(0.2, 0.8, (8, 3))
    x1 = x0 + rng.normal(0, 0.02, (8, 3))
    w = rng.normal(size=(8, cfg.in_dim))

    def f(th):
        p0 = O.inverse(th, x0)
        p1 = O.inverse(th, x1)
        return (O.encode_segments(cfg, tables, p0, p1) * w).sum()

    g = O.pose_gradient(cfg, tables, pose, O.inverse(pose, x0), O.inverse(pose, x1), w)
    # the cell coordinate is rounded to float32 (~6e-8), so the step must stay
    # large against that; the cells of this tiny grid are >= 1/4 wide
    h = 1e-3
    for j in range(3):
        e = np.zeros(3); e[j] = h
        fd = (f(pose + e) - f(pose - e)) / (2 * h)
        assert abs(fd - g[j]) <= 5e-3 * max(1.0, abs(fd)), (j, fd, g[j])


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(torch.bfloat16).to(torch.float64).numpy()


def test_rounded_mlp_reduces_to_exact_mlp():
    """With no rounding and unit scale the mixed-path MLP is the FP64 MLP
    (itself pinned by finite differences); the scale multiplies every
    gradient (linearity)."""
    rng = np.random.default_rng(14)
    ws = [rng.normal(size=sh) for sh in [(8, 10), (8, 8), (16, 8)]]
    x = rng.normal(size=(9, 10))
    dout = rng.normal(size=(9, 16))
    ident = lambda a: a
    out_r, acts_r = O.mlp_forward_rounded(ws, x, ident)
    out, acts = O.mlp_forward(ws, x)
    np.testing.assert_allclose(out_r, out, rtol=1e-13)
    dws, dx = O.mlp_backward(ws, acts, dout)
    for scale in (1.0, 1024.0):
        dws_r, dx_r = O.mlp_backward_rounded(ws, acts_r, dout, scale, ident)
        np.testing.assert_allclose(dx_r, scale * dx, rtol=1e-12)
        for a, b in zip(dws_r, dws):
            np.testing.assert_allclose(a, scale * b, rtol=1e-12)


def test_rounded_mlp_rounds_where_it_stores():
    """Hand-worked case in BF16 (8 significant bits, spacing 2^-7 in [1, 2)):
    one hidden unit, x = 1, W0 = 1 + 2^-9 -> 1, W1 = 3 + 2^-6 -> 3 (spacing
    2^-6 in [2, 4) keeps it: 3.015625). Forward: act = rnd(1 * 1) = 1, out =
    3.015625. Backward with dout = 1 + 2^-9 (-> 1) and scale 4: dY_1 = 4,
    dW1 = 4, dX = 4 * 3.015625 = 12.0625 -> rnd (spacing 2^-4 in [8, 16)) =
    12.0625, masked by act > 0; dW0 = 12.0625, dx = 12.0625 * 1."""
    ws = [np.array([[1 + 2.0 ** -9]]), np.array([[3 + 2.0 ** -6]])]
    out, acts = O.mlp_forward_rounded(ws, np.array([[1.0]]), _bf16)
    assert out[0, 0] == 3.015625 and acts[1][0, 0] == 1.0
    dws, dx = O.mlp_backward_rounded(ws, acts, np.array([[1 + 2.0 ** -9]]), 4.0, _bf16)
    assert dws[1][0, 0] == 4.0
    assert dws[0][0, 0] == 12.0625 and dx[0, 0] == 12.0625
    # a negative pre-activation: the ReLU mask zeroes the hidden gradient
    out, acts = O.mlp_forward_rounded([-ws[0], ws[1]], np.array([[1.0]]), _bf16)
    dws, dx = O.mlp_backward_rounded([-ws[0], ws[1]], acts, np.array([[1.0]]), 4.0, _bf16)
    assert out[0, 0] == 0.0 and dws[0][0, 0] == 0.0 and dx[0, 0] == 0.0 and dws[1][0, 0] == 0.0


# ---------------------------------------------------------------------------
# Curved-face reading of a deformed voxel: line / bilinear patch
# ---------------------------------------------------------------------------

def test_bilinear_patch_saddle_closed_form():
    """The patch x = u, y = v, z = u v (corners (0,0,0), (1,0,0), (0,1,0),
    (1,1,1)) meets the line x = s, y = 1 - s, z = c where s (1 - s) = c:
    s = (1 +- sqrt(1 - 4c)) / 2, two hits for 0 < c < 1/4, at (u, v) = (s, 1 - s)."""
    c = 0.16
    o = np.array([0.0, 1.0, c])
    d = np.array([1.0, -1.0, 0.0]) / math.sqrt(2.0)
    hits, sep = O.bilinear_hits(o, d, [0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 1])
    r = math.sqrt(1 - 4 * c)
    want = sorted([(1 - r) / 2, (1 + r) / 2])
    got = sorted(hits)
    assert len(got) == 2
    for (t, u, v), s in zip(got, want):
        assert abs(t - s * math.sqrt(2.0)) < 1e-14 and abs(u - s) < 1e-14 and abs(v - (1 - s)) < 1e-14
    assert abs(sep - r * math.sqrt(2.0)) < 1e-14
    # c > 1/4: the line passes above the saddle; c < 0: below the patch's z range at those (x, y)
    assert O.bilinear_hits(np.array([0.0, 1.0, 0.3]), d, [0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 1])[0] == []
    assert O.bilinear_hits(np.array([0.0, 1.0, -0.1]), d, [0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 1])[0] == []


def test_bilinear_patch_hits_constructed_points():
    """Lines built through a known point S(u0, v0) of random twisted patches
    must report that hit: t = t0, (u, v) = (u0, v0); swapping the u and v
    corners swaps (u, v); reversing d negates t."""
    rng = np.random.default_rng(61)
    for _ in range(300):
        P = rng.uniform(0, 1, (4, 3))
        u0, v0 = rng.uniform(0.05, 0.95, 2)
        S0 = P[0] + u0 * (P[1] - P[0]) + v0 * (P[2] - P[0]) + u0 * v0 * (P[3] - P[1] - P[2] + P[0])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        t0 = rng.uniform(0.5, 2.0)
        o = S0 - t0 * d
        hits, _ = O.bilinear_hits(o, d, *P)
        assert min(max(abs(t - t0), abs(u - u0), abs(v - v0)) for t, u, v in hits) < 1e-9
        sw, _ = O.bilinear_hits(o, d, P[0], P[2], P[1], P[3])
        assert min(max(abs(t - t0), abs(u - v0), abs(v - u0)) for t, u, v in sw) < 1e-9
        rv, _ = O.bilinear_hits(o, -d, *P)
        assert min(abs(t + t0) for t, _, _ in rv) < 1e-9


def test_bilinear_faces_equal_triangles_when_faces_are_planar():
    """At the identity pose every voxel hull is an axis-aligned cube whose
    faces are planar squares: the bilinear patch of a face and its two
    triangles are the same point set, so both readings give the same
    segments (voxels, counts and distances)."""
    N = 16
    occ, _, _ = O.voxelize(N, S.torus_mesh())
    rays = S.sphere_rays(2000, seed=62)
    a = O.segments(N, occ, (0.0, 0.0, 0.0), rays)
    b = O.segments(N, occ, (0.0, 0.0, 0.0), rays, faces="bilinear")
    np.testing.assert_array_equal(a.count, b.count)
    np.testing.assert_array_equal(a.vox, b.vox)
    np.testing.assert_allclose(b.t0, a.t0, atol=1e-12)
    np.testing.assert_allclose(b.t1, a.t1, atol=1e-12)
    # deformed: the same voxels on rays decided with margin, distances within the faces' bulge
    pose = (0.6, -0.8, 0.5)
    a = O.segments(N, occ, pose, rays)
    b = O.segments(N, occ, pose, rays, faces="bilinear")
    keep = np.nonzero((a.margin > 1e-3) & (b.margin > 1e-3))[0]
    assert len(keep) > 500
    for r in keep:
        np.testing.assert_array_equal(a.vox[a.off[r]:a.off[r + 1]], b.vox[b.off[r]:b.off[r + 1]])
        np.testing.assert_allclose(a.t0[a.off[r]:a.off[r + 1]], b.t0[b.off[r]:b.off[r + 1]], atol=0.02)
