"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Inputs come from the seeded generators only; the oracle never sees a value
produced by the GPU. Integer work (occupancy, triangle lists, voxel id
sequences, hash rows, labels' hit flags and materials) must match exactly
wherever the oracle's FP64 decision margin is clear of FP32 rounding; float
results match within the tolerances stated next to each assertion.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2604_24666_gb300 import synth as S
from tests import bounds as B
from tests.gpu_common import (LABEL_MARGIN, SEG_MARGIN, certain_rays, occupancy_biased_weights,
                              random_tables)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nif():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_24666_gb300 import nif as N
    N.lib()
    return N


@pytest.fixture(scope="module")
def torus():
    return S.torus_mesh()


@pytest.fixture(scope="module")
def ellipsoids():
    return S.ellipsoid_union_mesh()


def _dev():
    return torch.device("cuda:0")


# ---------------------------------------------------------------------------
# Voxelization (bit-exact)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,N", [("torus", 16), ("torus", 64), ("ellipsoids", 64)])
def test_voxelization_bit_exact(nif, torus, ellipsoids, shape, N):
    mesh = torus if shape == "torus" else ellipsoids
    net = S.NetConfig(voxel_res=N)
    h = nif.Nif(net, mesh)
    occ, ptr, idx = nif.nif_get_voxels(h.h, N)
    oocc, optr, oidx = O.voxelize(N, mesh)
    assert np.array_equal(occ, oocc)
    assert np.array_equal(ptr, optr)
    assert np.array_equal(idx, oidx)
    h.close()


# ---------------------------------------------------------------------------
# Segments (voxel sequences bit-exact on rays decided with margin)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("pose", [(0, 0, 0), (0.4, -0.7, 0.3), (-1.0, 1.0, -1.0), (1.0, -1.5, 1.0)])
def test_segments_match_oracle(nif, torus, pose):
    N = 16
    rays_np = S.sphere_rays(3000, seed=21)
    h = nif.Nif(S.NetConfig(voxel_res=N), torus)
    rays = torch.from_numpy(rays_np).to(_dev())
    offs, segs = nif.nif_segments(h.h, [pose], rays)
    off = offs.cpu().numpy().astype(np.int64)
    g = segs.cpu().numpy().view(nif.SEGMENT_DTYPE).reshape(-1)
    occ, _, _ = O.voxelize(N, torus)
    seg = O.segments(N, occ, pose, rays_np)
    certain = seg.margin > SEG_MARGIN
    assert certain.mean() > 0.97
    dt = []
    for r in np.nonzero(certain)[0]:
        gv = g[off[r]:off[r + 1]]
        a, b = seg.off[r], seg.off[r + 1]
        assert np.array_equal(gv["voxel"], seg.vox[a:b]), r
        assert np.all(gv["ray"] == r)
        dt.append(np.abs(gv["t0"] - seg.t0[a:b]))
        dt.append(np.abs(gv["t1"] - seg.t1[a:b]))
    dt = np.concatenate(dt)
    # FP32 hull corners (~5e-7) over the incidence cosine; grazing hits dominate the tail
    assert np.median(dt) < 1e-6 and dt.max() < 1e-3, (np.median(dt), dt.max())
    # every ray's list is sorted by (t0, voxel)
    for r in range(len(rays_np)):
        gv = g[off[r]:off[r + 1]]
        assert np.all(np.diff(gv["t0"]) >= 0)
    h.close()


def test_segments_multi_instance(nif, torus):
    N = 16
    poses = S.poses(5, seed=31)
    counts = [100, 0, 750, 1, 400]
    rays_np = S.sphere_rays(sum(counts), seed=32)
    inst = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    h = nif.Nif(S.NetConfig(voxel_res=N), torus)
    rays = torch.from_numpy(rays_np).to(_dev())
    offs, segs = nif.nif_segments(h.h, poses, rays, inst_offsets=torch.from_numpy(inst).to(_dev()))
    off = offs.cpu().numpy().astype(np.int64)
    g = segs.cpu().numpy().view(nif.SEGMENT_DTYPE).reshape(-1)
    occ, _, _ = O.voxelize(N, torus)
    n_cmp = 0
    for i in range(5):
        sub = rays_np[inst[i]:inst[i + 1]]
        if not len(sub):
            continue
        seg = O.segments(N, occ, poses[i], sub)
        for r in np.nonzero(seg.margin > SEG_MARGIN)[0]:
            R = inst[i] + r
            assert np.array_equal(g["voxel"][off[R]:off[R + 1]], seg.vox[seg.off[r]:seg.off[r + 1]])
            n_cmp += 1
    assert n_cmp > 1000
    h.close()


def test_segments_ellipsoids64(nif, ellipsoids):
    N = 64
    pose = (0.6, 0.9, -0.5)
    rays_np = S.sphere_rays(600, seed=33)
    h = nif.Nif(S.NetConfig(voxel_res=N), ellipsoids)
    offs, segs = nif.nif_segments(h.h, [pose], torch.from_numpy(rays_np).to(_dev()))
    off = offs.cpu().numpy().astype(np.int64)
    g = segs.cpu().numpy().view(nif.SEGMENT_DTYPE).reshape(-1)
    occ, _, _ = O.voxelize(N, ellipsoids)
    seg = O.segments(N, occ, pose, rays_np)
    certain = seg.margin > SEG_MARGIN
    assert certain.mean() > 0.8
    for r in np.nonzero(certain)[0]:
        assert np.array_equal(g["voxel"][off[r]:off[r + 1]], seg.vox[seg.off[r]:seg.off[r + 1]]), r
    h.close()


def test_empty_and_missing_rays(nif, torus):
    h = nif.Nif(S.NetConfig(voxel_res=16), torus)
    rays = torch.zeros((0, 8), dtype=torch.float32, device=_dev())
    offs, segs = nif.nif_segments(h.h, [(0, 0, 0)], rays)
    assert offs.shape[0] == 1 and int(offs[0]) == 0 and segs.shape[0] == 0
    # rays pointing away from the cube: no segments, no hits
    r = S.sphere_rays(64, seed=3)
    r[:, 3:6] *= -1
    rays = torch.from_numpy(r).to(_dev())
    offs, segs = nif.nif_segments(h.h, [(0.2, 0.2, 0.2)], rays)
    assert int(offs[-1]) == 0
    hits = nif.nif_query(h.h, [(0.2, 0.2, 0.2)], rays).cpu().numpy().view(nif.HIT_DTYPE).reshape(-1)
    assert not hits["hit"].any() and np.all(np.isinf(hits["D"]))
    h.close()


# ---------------------------------------------------------------------------
# Linearization
# ---------------------------------------------------------------------------
def test_linearize_matches_oracle(nif, torus):
    N = 16
    pose = (0.8, -1.2, 0.6)
    rays_np = S.sphere_rays(1000, seed=41)
    keep = certain_rays(N, torus, pose, rays_np)
    rays_np = rays_np[keep]
    h = nif.Nif(S.NetConfig(voxel_res=N), torus)
    rays = torch.from_numpy(rays_np).to(_dev())
    offs, segs = nif.nif_segments(h.h, [pose], rays)
    lin = nif.nif_linearize(h.h, [pose], rays, segs).cpu().numpy().view(nif.LINSEG_DTYPE).reshape(-1)
    occ, _, _ = O.voxelize(N, torus)
    seg = O.segments(N, occ, pose, rays_np)
    p0, p1, ld, lr = O.linearize(pose, rays_np, seg)
    assert len(lin) == len(seg)
    # t errors (<= ~1e-4 on grazing faces) times |dD^-1/dx| (<= ~2)
    np.testing.assert_allclose(lin["p0"], p0, atol=5e-4)
    np.testing.assert_allclose(lin["p1"], p1, atol=5e-4)
    assert np.median(np.abs(lin["p0"] - p0)) < 2e-6
    np.testing.assert_allclose(lin["l_def"], ld, atol=5e-4)
    np.testing.assert_allclose(lin["l_rest"], lr, atol=1e-3)
    h.close()


# ---------------------------------------------------------------------------
# Encoding
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("levels,log2T", [(8, 14), (16, 19)])
def test_encode_points_rows_and_features(nif, torus, levels, log2T):
    net = S.NetConfig(levels=levels, log2_table=log2T)
    h = nif.Nif(net, torus)
    tables = random_tables(net, 51)
    h.set_params(tables, S.init_params(net)[1])
    rng = np.random.default_rng(52)
    pts = rng.uniform(-0.05, 1.05, (3000, 3)).astype(np.float32)
    pts[:8] = [[0, 0, 0], [1, 1, 1], [0.5, 0.5, 0.5], [1, 0, 1], [0.25, 0.75, 0.125], [0.999999, 0, 0.5],
               [1e-7, 0.5, 1], [0.5, 1, 0]]
    width = net.n_terms * levels * 2
    f, rows = nif.nif_encode_points(h.h, torch.from_numpy(pts).to(_dev()), width, rows=True,
                                    n_terms=net.n_terms, levels=levels)
    f = f.cpu().numpy().reshape(len(pts), net.n_terms, levels, 2)
    rows = rows.cpu().numpy().reshape(len(pts), net.n_terms, levels)
    ref = O.encode_points(net, tables, pts.astype(np.float64)).reshape(len(pts), net.n_terms, levels, 2)
    _, u = O.gamma(net, pts.astype(np.float64))
    res = O.level_res(net)
    mism = 0
    for t in range(net.n_terms):
        for l in range(levels):
            i0, w = O._cell(net, l, u[:, t])
            orow = O.grid_index(net, l, i0)
            if t == 0:
                # identical float32 u on both sides: bit-exact rows
                assert np.array_equal(rows[:, t, l], orow), (t, l)
            else:
                # u = (sin+1)/2 differs by a few ulps: rows differ only at cell faces
                bad = rows[:, t, l] != orow
                q = (u[:, t] * res[l])
                near = np.abs(q - np.round(q)).min(axis=1) < 2e-6 * res[l] + 1e-6
                assert np.all(near[bad]), (t, l)
                mism += bad.sum()
            du = 0.0 if t == 0 else 4e-7
            tol = 2e-6 + 8 * res[l] * du * 2
            np.testing.assert_allclose(f[:, t, l], ref[:, t, l], atol=tol, rtol=0)
    assert mism < 0.001 * rows.size
    h.close()


def test_encode_points_backward(nif, torus):
    """Table gradient entry by entry and dL/dp point by point against the
    bounds of tests/bounds.py (points whose cells FP32 could move are left
    out before either side runs)."""
    net = S.NetConfig(levels=8, log2_table=12)
    h = nif.Nif(net, torus)
    tables = random_tables(net, 61)
    h.set_params(tables, S.init_params(net)[1])
    rng = np.random.default_rng(62)
    pts = rng.uniform(0.02, 0.98, (2400, 3)).astype(np.float32)
    pts = pts[B.certain_cells(net, pts)][:2000]
    assert len(pts) == 2000
    width = net.n_terms * net.levels * 2
    df = rng.normal(size=(len(pts), width)).astype(np.float32)
    dtab = torch.zeros((net.levels, 1 << net.log2_table, 2), dtype=torch.float32, device=_dev())
    dp = nif.nif_encode_points_backward(h.h, torch.from_numpy(pts).to(_dev()), torch.from_numpy(df).to(_dev()), dtab)
    p64, d64 = pts.astype(np.float64), df.astype(np.float64)
    rt, rp = O.encode_points_backward(net, tables, p64, d64)
    g = dtab.cpu().numpy()
    bt = B.table_grad_bound(net, tables, p64, d64)
    assert np.all(np.abs(g - rt) <= bt), (np.abs(g - rt) / np.maximum(bt, 1e-300)).max()
    gp = dp.cpu().numpy()
    bp = B.point_grad_bound(net, tables, p64, d64)
    assert np.all(np.abs(gp - rp) <= bp), (np.abs(gp - rp) / np.maximum(bp, 1e-300)).max()
    h.close()


@pytest.mark.parametrize("levels", [12, 6])
def test_deterministic_table_gradient_other_level_counts(nif, torus, levels):
    """NIF_KNOB_DETERMINISTIC on handles whose level count does not divide
    32 (one thread per segment end point and gamma term, every contribution
    rounded to 64-bit fixed point alone): the table gradient of the segment
    encoding repeats bit for bit and meets the oracle's bound plus 2^-(S+1)
    per contribution, entry by entry."""
    net = S.NetConfig(levels=levels, log2_table=12)
    h = nif.Nif(net, torus)
    tables = random_tables(net, 71)
    h.set_params(tables, S.init_params(net)[1])
    lin, _ = S.chained_segments(3000, seed=72, voxel_res=net.voxel_res, gap=0.1)
    keep = B.certain_cells(net, lin[:, 0:3]) & B.certain_cells(net, lin[:, 3:6])
    lin = lin[keep][:2000]
    n = len(lin)
    assert n == 2000
    df = np.random.default_rng(73).normal(size=(n, net.in_dim)).astype(np.float32)
    lint, dft = torch.from_numpy(lin).to(_dev()), torch.from_numpy(df).to(_dev())
    nif.nif_set_knob(h.h, nif.NIF_KNOB_DETERMINISTIC, 1)
    runs = []
    for _ in range(2):
        d = torch.zeros((net.levels, 1 << net.log2_table, 2), dtype=torch.float32, device=_dev())
        nif.nif_encode_segments_backward(h.h, lint, dft, d)
        runs.append(d)
    torch.cuda.synchronize()
    assert torch.equal(runs[0], runs[1])
    g = runs[0].cpu().numpy()
    half = net.in_dim // 2
    p = np.concatenate([lin[:, 0:3], lin[:, 3:6]]).astype(np.float64)
    d = np.concatenate([df[:, :half], df[:, half:]]).astype(np.float64)
    ref, _ = O.encode_points_backward(net, tables, p, d)
    bnd = B.table_grad_bound(net, tables, p, d, fix_S=B.fixed_scale(n, net.n_terms, df))
    err = np.abs(g - ref)
    assert np.all(err <= bnd), ((err / np.maximum(bnd, 1e-300)).max(), int((err > bnd).sum()))
    h.close()


# ---------------------------------------------------------------------------
# MLP (FP32)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fused", [0, 1])
@pytest.mark.parametrize("depth,width,levels", [(2, 32, 8), (3, 64, 16)])
def test_mlp_fp32_forward_backward(nif, torus, depth, width, levels, fused):
    """Per-layer launches (fused = 0) and the one-launch forward (fused = 1)."""
    net = S.NetConfig(levels=levels, log2_table=14, mlp_depth=depth, mlp_width=width)
    h = nif.Nif(net, torus)
    nif.nif_set_knob(h.h, nif.NIF_KNOB_FP32_FUSED, fused)
    tables, ws, s = S.init_params(net, seed=71)
    h.set_params(tables, ws, s)
    rng = np.random.default_rng(72)
    n = 1000 + 37                       # several tiles and a ragged tail
    x = rng.normal(size=(n, net.in_dim)).astype(np.float32)
    xt = torch.from_numpy(x).to(_dev())
    acts = torch.zeros((depth, n, width), dtype=torch.float32, device=_dev())
    out = nif.nif_mlp_forward(h.h, xt, acts=acts).cpu().numpy()
    ref, racts = O.mlp_forward(ws, x.astype(np.float64))
    scale = np.abs(ref).max()
    np.testing.assert_allclose(out, ref, atol=2e-5 * scale)
    dout = rng.normal(size=(n, 16)).astype(np.float32)
    dout[:, net.out_dim:] = 0
    nif.nif_zero_grad(h.h)
    dx = nif.nif_mlp_backward(h.h, xt, acts, torch.from_numpy(dout).to(_dev())).cpu().numpy()
    torch.cuda.synchronize()
    rdw, rdx = O.mlp_backward(ws, racts, dout.astype(np.float64))
    np.testing.assert_allclose(dx, rdx, atol=2e-5 * np.abs(rdx).max())
    _, gws, _ = h.get_grads()
    for gw, rw in zip(gws, rdw):
        np.testing.assert_allclose(gw, rw, atol=2e-5 * np.abs(rw).max() + 1e-7)
    h.close()


# ---------------------------------------------------------------------------
# Labels and losses
# ---------------------------------------------------------------------------
def _labels_inputs(nif, mesh, N, pose, n_rays, seed):
    rays_np = S.sphere_rays(n_rays, seed=seed)
    keep = certain_rays(N, mesh, pose, rays_np, with_labels=True)
    return rays_np[keep]


def test_labels_match_oracle(nif, torus):
    N = 16
    pose = (0.5, 1.0, -0.5)
    rays_np = _labels_inputs(nif, torus, N, pose, 2000, 81)
    h = nif.Nif(S.NetConfig(voxel_res=N), torus)
    rays = torch.from_numpy(rays_np).to(_dev())
    offs, segs = nif.nif_segments(h.h, [pose], rays)
    lin = nif.nif_linearize(h.h, [pose], rays, segs)
    lab = nif.nif_labels(h.h, segs, lin).cpu().numpy().view(nif.LABEL_DTYPE).reshape(-1)
    occ, ptr, idx = O.voxelize(N, torus)
    seg = O.segments(N, occ, pose, rays_np)
    p0, p1, ld, lr = O.linearize(pose, rays_np, seg)
    ref = O.labels(torus, ptr, idx, seg.vox, p0, p1)
    assert np.array_equal(lab["occ"], ref["occ"])
    hit = ref["occ"] == 1
    assert hit.sum() > 200
    assert np.array_equal(lab["material"][hit], ref["material"][hit])
    np.testing.assert_allclose(lab["tpar"][hit], ref["tpar"][hit], atol=2e-3)
    np.testing.assert_allclose(lab["normal"][hit], ref["normal"][hit], atol=1e-5)
    np.testing.assert_allclose(lab["albedo"][hit], ref["albedo"][hit], atol=0)
    h.close()


@pytest.mark.parametrize("flags", [0, 1, 2, 3])
def test_loss_matches_oracle(nif, torus, flags):
    net = S.NetConfig()
    h = nif.Nif(net, torus, flags=flags)
    rng = np.random.default_rng(91)
    n = 3001
    out = rng.normal(size=(n, 16)).astype(np.float32)
    out[:, 12:] = 0
    occ = (rng.random(n) < 0.4).astype(np.uint8)
    nrm = rng.normal(size=(n, 3)); nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    lab = np.zeros(n, dtype=nif.LABEL_DTYPE)
    lab["tpar"] = rng.uniform(0, 1, n)
    lab["normal"] = nrm
    lab["albedo"] = rng.uniform(0, 1, (n, 3))
    lab["occ"] = occ
    lab["material"] = rng.integers(0, 4, n)
    lin = np.zeros(n, dtype=nif.LINSEG_DTYPE)
    lin["l_rest"] = rng.uniform(0.2, 1.5, n) / net.voxel_res
    s = np.array([0.3, -0.2, 0.1, 0.5, -0.4], np.float32)
    h.set_params(*S.init_params(net)[:2], s)
    nif.nif_zero_grad(h.h)
    labt = torch.from_numpy(lab.view(np.float32).reshape(n, 8).copy()).to(_dev())
    lint = torch.from_numpy(lin.view(np.float32).reshape(n, 8).copy()).to(_dev())
    parts, dout = nif.nif_loss(h.h, torch.from_numpy(out).to(_dev()), labt, lint)
    ds = h.get_grads()[2]
    rl = dict(occ=lab["occ"], tpar=lab["tpar"].astype(np.float64), normal=lab["normal"].astype(np.float64),
              albedo=lab["albedo"].astype(np.float64), material=lab["material"])
    tot, rparts, rdout, rds = O.loss(net, out.astype(np.float64), rl, s.astype(np.float64),
                                     lin["l_rest"].astype(np.float64), flags)
    np.testing.assert_allclose(parts[1:], rparts, rtol=1e-5)
    assert abs(parts[0] - tot) < 1e-5 * max(1, abs(tot))
    np.testing.assert_allclose(dout.cpu().numpy(), rdout, atol=1e-5 * np.abs(rdout).max())
    np.testing.assert_allclose(ds[:5], rds, atol=1e-5)
    h.close()


# ---------------------------------------------------------------------------
# Whole query
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("pose,fused", [((0, 0, 0), 1), ((0.6, -1.0, 0.4), 1), ((0.6, -1.0, 0.4), 0)])
def test_query_fp32_matches_oracle(nif, torus, pose, fused):
    """fused: the MLP forward in one launch, which stores no hidden
    activations in a query (NIF_KNOB_FP32_FUSED, default), or one launch per
    layer."""
    net = S.NetConfig()
    h = nif.Nif(net, torus)
    nif.nif_set_knob(h.h, nif.NIF_KNOB_FP32_FUSED, fused)
    tables = random_tables(net, 101)
    ws, s = occupancy_biased_weights(net, 102)
    h.set_params(tables, ws, s)
    rays_np = S.sphere_rays(1500, seed=103)
    keep = certain_rays(net.voxel_res, torus, pose, rays_np)
    rays_np = rays_np[keep]
    hits = nif.nif_query(h.h, [pose], torch.from_numpy(rays_np).to(_dev())).cpu().numpy()
    hits = hits.view(nif.HIT_DTYPE).reshape(-1)
    occ, _, _ = O.voxelize(net.voxel_res, torus)
    seg = O.segments(net.voxel_res, occ, pose, rays_np)
    p0, p1, ld, lr = O.linearize(pose, rays_np, seg)
    out = O.mlp_forward(ws, O.encode_segments(net, tables, p0, p1))[0]
    res = O.reconstruct(net, pose, rays_np, seg, out, p0, p1, ld, lr)
    n_cmp = 0
    for r in range(len(rays_np)):
        a, b = seg.off[r], seg.off[r + 1]
        if np.any(np.abs(out[a:b, 0]) < 1e-3):
            continue                                # occupancy decision too close to call
        assert hits["hit"][r] == res["hit"][r], r
        if res["hit"][r]:
            j = a + res["k"][r]
            if np.abs(out[j, 8:12] - out[j, 8:12].max()).__lt__(1e-3).sum() == 1:
                assert hits["material"][r] == res["material"][r]
            assert abs(hits["D"][r] - res["D"][r]) < 2e-4, (r, hits["D"][r], res["D"][r])
            np.testing.assert_allclose(hits["albedo"][r], res["albedo"][r], atol=1e-4)
            assert np.dot(hits["n"][r], res["normal"][r]) > np.cos(np.radians(0.05))
        n_cmp += 1
    assert n_cmp > 800
    assert hits["hit"].sum() > 100
    h.close()


# ---------------------------------------------------------------------------
# Gradients of a training batch and Adam
# ---------------------------------------------------------------------------
def _certain_loss_rows(net, ws, x, lab):
    """Rows whose every branch (hidden ReLUs, the distance head's ReLU, the
    albedo L1's sign) FP32 and FP64 take alike."""
    ok = B.relu_certain_rows(ws, x)
    out, _ = O.mlp_forward(ws, x)
    hit = lab["occ"] == 1
    zd = out[:, 1]
    ok &= ~hit | (np.abs(zd) > 1e-4 * np.abs(zd).max())
    alb = 0.5 * (1.0 + np.tanh(0.5 * out[:, 5:8]))
    ok &= ~hit | (np.abs(alb - lab["albedo"]).min(axis=1) > 1e-5)
    return ok


def _abs_mat(ws, lo, hi):
    """|W_{hi-1}| ... |W_lo|: how an error at the output of layer hi-1 can grow
    back to the input of layer lo (ReLU masks only shrink it)."""
    m = np.abs(np.asarray(ws[hi - 1], np.float64))
    for i in range(hi - 2, lo - 1, -1):
        m = m @ np.abs(np.asarray(ws[i], np.float64))
    return m


@pytest.mark.parametrize("det", [0, 1], ids=["l2-reductions", "deterministic"])
def test_train_gradients_match_oracle(nif, torus, det):
    """The whole backward of a training batch (loss -> MLP backward ->
    encoding backward -> parameter gradients) on identical inputs: linearized
    segments from the seeded generator, ground-truth labels from the oracle
    (fed to both sides), so that every gradient can be compared element by
    element. Bounds: loss output gradient 1e-5 of its largest entry (FP32
    loss), carried back through |W| (tests/bounds.py for the encoding). With
    NIF_KNOB_DETERMINISTIC the table gradient's bound adds the fixed-point
    rounding, 2^-(S+1) per contribution, and a second backward on the same
    inputs must give the same gradients bit for bit."""
    net = S.NetConfig()
    N = net.voxel_res
    occ, ptr, idx = O.voxelize(N, torus)
    lin, vox = S.chained_segments(24000, seed=111, voxel_res=N, gap=0.1)
    keep = (occ.reshape(-1)[vox] == 1) & B.certain_cells(net, lin[:, 0:3]) & B.certain_cells(net, lin[:, 3:6])
    lin, vox = lin[keep], vox[keep]
    tables = random_tables(net, 112, scale=0.5)
    _, ws, _ = S.init_params(net, seed=113)
    s = np.array([0.1, -0.1, 0.2, 0.0, 0.3], np.float32)
    p0, p1 = lin[:, 0:3].astype(np.float64), lin[:, 3:6].astype(np.float64)
    rlab = O.labels(torus, ptr, idx, vox, p0, p1)
    x = O.encode_segments(net, tables, p0, p1)
    keep = _certain_loss_rows(net, ws, x, rlab)
    lin, vox, p0, p1, x = lin[keep], vox[keep], p0[keep], p1[keep], x[keep]
    rlab = {k: v[keep] for k, v in rlab.items()}
    n = len(lin)
    assert n > 1500 and rlab["occ"].sum() > 300, (n, rlab["occ"].sum())

    h = nif.Nif(net, torus)
    if det:
        nif.nif_set_knob(h.h, nif.NIF_KNOB_DETERMINISTIC, 1)
    h.set_params(tables, ws, s)
    lab = np.zeros(n, dtype=nif.LABEL_DTYPE)
    for k in ("tpar", "normal", "albedo", "occ", "material"):
        lab[k] = rlab[k]
    labt = torch.from_numpy(lab.view(np.float32).reshape(n, 8).copy()).to(_dev())
    lint = torch.from_numpy(lin).to(_dev())
    feat = nif.nif_encode_segments(h.h, lint, net.in_dim)
    acts = torch.zeros((net.mlp_depth, n, net.mlp_width), dtype=torch.float32, device=_dev())
    out = nif.nif_mlp_forward(h.h, feat, acts=acts)
    nif.nif_zero_grad(h.h)
    parts, dout = nif.nif_loss(h.h, out, labt, lint)
    dx = nif.nif_mlp_backward(h.h, feat, acts, dout)
    dtab = torch.zeros((net.levels, 1 << net.log2_table, 2), dtype=torch.float32, device=_dev())
    nif.nif_encode_segments_backward(h.h, lint, dx, dtab)
    torch.cuda.synchronize()
    _, gws, gs = h.get_grads()
    if det:
        # the same backward again: every gradient repeats bit for bit
        nif.nif_zero_grad(h.h)
        parts2, dout2 = nif.nif_loss(h.h, out, labt, lint)
        dx2 = nif.nif_mlp_backward(h.h, feat, acts, dout2)
        dtab2 = torch.zeros_like(dtab)
        nif.nif_encode_segments_backward(h.h, lint, dx2, dtab2)
        torch.cuda.synchronize()
        _, gws2, gs2 = h.get_grads()
        assert np.array_equal(parts2, parts)
        assert torch.equal(dx2, dx) and torch.equal(dtab2, dtab)
        assert all(np.array_equal(a, b) for a, b in zip(gws2, gws)) and np.array_equal(gs2, gs)
    fix_S = B.fixed_scale(n, net.n_terms, dx.cpu().numpy()) if det else None
    dout, dx, g = dout.cpu().numpy(), dx.cpu().numpy(), dtab.cpu().numpy()

    o, racts = O.mlp_forward(ws, x)
    tot, rparts, rdout, rds = O.loss(net, o, rlab, s, lin[:, 7].astype(np.float64))
    rdw, rdx = O.mlp_backward(ws, racts, rdout)
    half = net.in_dim // 2
    rt = O.encode_points_backward(net, tables, np.concatenate([p0, p1]),
                                  np.concatenate([rdx[:, :half], rdx[:, half:]]))[0]
    assert abs(parts[0] - tot) < 1e-5 * max(1.0, abs(tot))
    np.testing.assert_allclose(parts[1:], rparts, rtol=1e-5)
    # the outputs carry the FP32 MLP's error (its bar: 2e-5 of the largest
    # output); the loss gradient moves with them, most near a zero distance
    # prediction, where the log loss's curvature is 1/(d + eps)^2
    out_err = np.full(o.shape[1], 2e-5 * np.abs(o).max())
    rnd = (1e-5 * np.abs(rdout) + 1e-6 * np.abs(rdout).max()) * (rdout != 0)   # FP32 loss arithmetic
    e_out = rnd + B.loss_grad_bound(net, o, rlab, s, lin[:, 7].astype(np.float64), out_err)
    assert np.all(np.abs(dout - rdout) <= e_out), (np.abs(dout - rdout) / e_out).max()
    np.testing.assert_allclose(gs[:5], rds, atol=1e-4)
    L = len(ws)
    # |dY_l| errors carried back through |W|: row-wise
    tol_dx = 2e-5 * np.abs(rdx).max() + e_out @ _abs_mat(ws, 0, L)
    assert np.all(np.abs(dx - rdx) <= tol_dx), (np.abs(dx - rdx) / tol_dx).max()
    for i in range(L):
        ey = e_out @ _abs_mat(ws, i + 1, L) if i + 1 < L else e_out
        tol = 2e-5 * np.abs(rdw[i]).max() + ey.T @ np.abs(racts[i])
        assert np.all(np.abs(gws[i] - rdw[i]) <= tol), (i, (np.abs(gws[i] - rdw[i]) / tol).max())
    bt = B.table_grad_bound(net, tables, np.concatenate([p0, p1]), np.concatenate([rdx[:, :half], rdx[:, half:]]),
                            dfeat_err=np.concatenate([tol_dx[:, :half], tol_dx[:, half:]]), fix_S=fix_S)
    assert np.all(np.abs(g - rt) <= bt), (np.abs(g - rt) / np.maximum(bt, 1e-300)).max()
    h.close()


def test_adam_matches_oracle(nif, torus):
    net = S.NetConfig(levels=4, log2_table=10)
    h = nif.Nif(net, torus)
    tables, ws, s = S.init_params(net, seed=121)
    s = np.array([0.1, 0.2, -0.3, 0.4, 0.0], np.float32)
    h.set_params(tables, ws, s)
    rng = np.random.default_rng(122)
    groups = [(nif.NIF_PARAM_TABLES, tables, 1e-2), (nif.NIF_PARAM_LOGVAR, s, 1e-2)] + \
             [(nif.NIF_PARAM_LAYER0 + i, w, 1e-3) for i, w in enumerate(ws)]
    state = {g: (p.astype(np.float64).ravel(), np.zeros(p.size), np.zeros(p.size)) for g, p, _ in groups}
    for step in (1, 2, 3):
        for g, p, lr in groups:
            gr = (rng.normal(size=p.size) * (rng.random(p.size) < 0.5)).astype(np.float32)
            if g == nif.NIF_PARAM_LAYER0 + len(ws) - 1:
                gr.reshape(p.shape)[net.out_dim:] = 0
            nif.nif_set_grad(h.h, g, gr)
            th, m, v = state[g]
            state[g] = O.adam(th, m, v, gr.astype(np.float64), step, lr)
        nif.nif_adam_step(h.h, 1e-2, 1e-3)
        torch.cuda.synchronize()
        for g, p, lr in groups:
            got = nif.nif_get_params(h.h, g)
            np.testing.assert_allclose(got, state[g][0], atol=1e-6 + 1e-6 * lr * 100)
            assert not nif.nif_get_grad(h.h, g).any()     # Adam clears the gradient
    h.close()


# ---------------------------------------------------------------------------
# Tensor-core MLP (BF16 / FP16 operands, FP32 accumulation)
# ---------------------------------------------------------------------------
def _quant(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).to(torch.float64).numpy()


def _mlp_lowp_reference(ws, x, dt):
    """FP64 MLP on 16-bit-rounded inputs and weights, hidden activations rounded
    to the same 16-bit type after the ReLU (as the kernel stores them)."""
    h = _quant(x, dt)
    for i, w in enumerate(ws):
        z = h @ _quant(w, dt).T
        if i < len(ws) - 1:
            h = _quant(np.maximum(z, 0.0), dt)
        else:
            h = z
    return h


@pytest.mark.parametrize("depth,width,levels", [(2, 32, 8), (3, 64, 16), (1, 128, 8)])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_mlp_tensor_core_forward(nif, torus, depth, width, levels, prec):
    net = S.NetConfig(levels=levels, log2_table=14, mlp_depth=depth, mlp_width=width)
    dt = torch.bfloat16 if prec == "bf16" else torch.float16
    p = nif.NIF_BF16 if prec == "bf16" else nif.NIF_FP16
    h = nif.Nif(net, torus)
    tables, ws, s = S.init_params(net, seed=131)
    h.set_params(tables, ws, s)
    rng = np.random.default_rng(132)
    for n in (1, 128, 5 * 128 + 77, 40000):     # one row, one tile, ragged tail, many tiles per CTA
        x = rng.normal(size=(n, net.in_dim)).astype(np.float32)
        xt = torch.from_numpy(x).to(_dev()).to(dt)
        out = nif.nif_mlp_forward(h.h, xt, precision=p).cpu().numpy()
        ref = _mlp_lowp_reference(ws, x, dt)
        scale = np.abs(ref).max()
        err = np.abs(out - ref)
        # FP32 accumulation vs FP64, plus rare one-ulp flips of rounded hidden activations
        assert np.median(err) <= 1e-4 * scale, (n, np.median(err), scale)
        assert err.max() <= 2e-2 * scale, (n, err.max(), scale)
        assert np.all(out[:, net.out_dim:] == 0)
    h.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_query_mixed_precision_error_vs_oracle(nif, torus, prec):
    """FP16 tables + 16-bit MLP operands against the FP64 oracle on the same
    weights. Bounds (stated, generous against the measured values): hit
    agreement on rays whose occupancy logit is clear of 5 % of its range,
    distance <= 2e-3, albedo <= 2e-2, normal within 2 degrees, material
    agreement >= 99 % where the top two logits differ by > 5 % of the range."""
    net = S.NetConfig()
    p = nif.NIF_BF16 if prec == "bf16" else nif.NIF_FP16
    h = nif.Nif(net, torus, precision=p)
    tables = random_tables(net, 141)
    ws, s = occupancy_biased_weights(net, 142)
    h.set_params(tables, ws, s)
    pose = (0.5, -0.8, 0.4)
    rays_np = S.sphere_rays(2000, seed=143)
    rays_np = rays_np[certain_rays(net.voxel_res, torus, pose, rays_np)]
    hits = nif.nif_query(h.h, [pose], torch.from_numpy(rays_np).to(_dev())).cpu().numpy()
    hits = hits.view(nif.HIT_DTYPE).reshape(-1)
    occ, _, _ = O.voxelize(net.voxel_res, torus)
    seg = O.segments(net.voxel_res, occ, pose, rays_np)
    p0, p1, ld, lr = O.linearize(pose, rays_np, seg)
    out = O.mlp_forward(ws, O.encode_segments(net, tables, p0, p1))[0]
    res = O.reconstruct(net, pose, rays_np, seg, out, p0, p1, ld, lr)
    zr = np.abs(out[:, 0]).max()
    n_cmp, mat_ok, mat_n = 0, 0, 0
    for r in range(len(rays_np)):
        a, b = seg.off[r], seg.off[r + 1]
        if np.any(np.abs(out[a:b, 0]) < 0.05 * zr):
            continue
        assert hits["hit"][r] == res["hit"][r], r
        if res["hit"][r]:
            j = a + res["k"][r]
            assert abs(hits["D"][r] - res["D"][r]) < 2e-3, (r, hits["D"][r], res["D"][r])
            np.testing.assert_allclose(hits["albedo"][r], res["albedo"][r], atol=2e-2)
            assert np.dot(hits["n"][r], res["normal"][r]) > np.cos(np.radians(2.0))
            m = np.sort(out[j, 8:12])
            if m[-1] - m[-2] > 0.05 * (np.abs(out[:, 8:12]).max()):
                mat_n += 1
                mat_ok += hits["material"][r] == res["material"][r]
        n_cmp += 1
    assert n_cmp > 500
    assert mat_n == 0 or mat_ok >= 0.99 * mat_n
    h.close()


# ---------------------------------------------------------------------------
# Differentiation: autograd over the library, gradients w.r.t. the pose
# ---------------------------------------------------------------------------
def test_autograd_function_matches_oracle(nif, torus):
    from paper_2604_24666_gb300.autograd import nif_segments_forward
    net = S.NetConfig(levels=8, log2_table=12)
    h = nif.Nif(net, torus)
    tables = random_tables(net, 151, scale=0.5)
    _, ws, s = S.init_params(net, seed=152)
    h.set_params(tables, ws, s)
    nif.nif_zero_grad(h.h)
    rng = np.random.default_rng(153)
    m = 1000
    p0 = rng.uniform(0.05, 0.95, (m, 3)).astype(np.float32)
    p1 = np.clip(p0 + rng.normal(0, 0.03, (m, 3)), 0.01, 0.99).astype(np.float32)
    ok = B.certain_cells(net, p0) & B.certain_cells(net, p1)
    ok &= B.relu_certain_rows(ws, O.encode_segments(net, tables, p0.astype(np.float64), p1.astype(np.float64)))
    p0, p1 = p0[ok][:700], p1[ok][:700]
    n = len(p0)
    assert n == 700
    wout = rng.normal(size=(n, 16)).astype(np.float32)
    wout[:, net.out_dim:] = 0
    t0 = torch.from_numpy(p0).to(_dev()).requires_grad_(True)
    t1 = torch.from_numpy(p1).to(_dev()).requires_grad_(True)
    out = nif_segments_forward(t0, t1, h)
    (out * torch.from_numpy(wout).to(_dev())).sum().backward()
    torch.cuda.synchronize()
    q0, q1 = p0.astype(np.float64), p1.astype(np.float64)
    x = O.encode_segments(net, tables, q0, q1)
    ro, racts = O.mlp_forward(ws, x)
    np.testing.assert_allclose(out.detach().cpu().numpy(), ro, atol=2e-5 * np.abs(ro).max())
    rdw, rdx = O.mlp_backward(ws, racts, wout.astype(np.float64))
    half = net.in_dim // 2
    e_dx = 2e-5 * np.abs(rdx).max()             # the FP32 MLP backward's bar
    rt0, rp0 = O.encode_points_backward(net, tables, q0, rdx[:, :half])
    rt1, rp1 = O.encode_points_backward(net, tables, q1, rdx[:, half:])
    for got, ref, q, d in ((t0.grad, rp0, q0, rdx[:, :half]), (t1.grad, rp1, q1, rdx[:, half:])):
        b = B.point_grad_bound(net, tables, q, d, dfeat_err=e_dx)
        err = np.abs(got.cpu().numpy() - ref)
        assert np.all(err <= b), (err / np.maximum(b, 1e-300)).max()
    gt, gws, _ = h.get_grads()
    bt = B.table_grad_bound(net, tables, np.concatenate([q0, q1]),
                            np.concatenate([rdx[:, :half], rdx[:, half:]]), dfeat_err=e_dx)
    assert np.all(np.abs(gt - (rt0 + rt1)) <= bt), (np.abs(gt - (rt0 + rt1)) / np.maximum(bt, 1e-300)).max()
    for a, b in zip(gws, rdw):
        np.testing.assert_allclose(a, b, atol=2e-5 * np.abs(b).max(), rtol=0)
    h.close()


def test_pose_gradient_matches_oracle(nif, torus):
    net = S.NetConfig(levels=8, log2_table=12)
    N = net.voxel_res
    poses = np.array([[0.5, -0.9, 0.4], [-0.7, 0.6, -0.3]], np.float32)
    parts = []
    for i, seed in enumerate((161, 164)):
        r = S.sphere_rays(700, seed=seed)
        parts.append(r[certain_rays(N, torus, poses[i], r)])   # identical segment lists on both sides
    rays_np = np.concatenate(parts)
    inst = np.array([0, len(parts[0]), len(rays_np)], np.int32)
    h = nif.Nif(net, torus)
    tables = random_tables(net, 162, scale=0.5)
    h.set_params(tables, S.init_params(net)[1])
    rays = torch.from_numpy(rays_np).to(_dev())
    it = torch.from_numpy(inst).to(_dev())
    offs, segs = nif.nif_segments(h.h, poses, rays, inst_offsets=it)
    lin = nif.nif_linearize(h.h, poses, rays, segs, inst_offsets=it)
    n = segs.shape[0]
    rng = np.random.default_rng(163)
    df = rng.normal(size=(n, net.in_dim)).astype(np.float32)
    dposes = nif.nif_pose_gradient(h.h, poses, segs, lin, torch.from_numpy(df).to(_dev()), inst_offsets=it)
    torch.cuda.synchronize()
    occ, _, _ = O.voxelize(N, torus)
    ref = np.zeros((2, 3))
    start = 0
    for i in range(2):
        seg = O.segments(N, occ, poses[i], parts[i])
        p0, p1, _, _ = O.linearize(poses[i], parts[i], seg)
        ref[i] = O.pose_gradient(net, tables, poses[i], p0, p1, df[start:start + len(seg)].astype(np.float64))
        start += len(seg)
    assert start == n
    np.testing.assert_allclose(dposes.cpu().numpy(), ref, rtol=5e-3, atol=5e-3 * np.abs(ref).max())
    h.close()


# ---------------------------------------------------------------------------
# Batched query captured as a CUDA graph
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_query_plan_graph_replays_match_query(nif, torus, prec):
    net = S.NetConfig()
    p = nif.NIF_BF16 if prec == "bf16" else nif.NIF_FP32
    h = nif.Nif(net, torus, precision=p)
    tables = random_tables(net, 171)
    ws, s = occupancy_biased_weights(net, 172)
    h.set_params(tables, ws, s)
    counts = [900, 0, 1300, 17]
    inst = torch.from_numpy(np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)).to(_dev())
    rays = torch.from_numpy(S.sphere_rays(sum(counts), seed=173)).to(_dev())
    hits = torch.zeros((sum(counts), 8), dtype=torch.float32, device=_dev())
    poses_a = S.poses(4, seed=174)
    poses_b = S.poses(4, seed=175)
    plan = nif.QueryPlan(h.h, poses_a, rays, hits, inst_offsets=inst, autotune=True)
    knobs = plan.info()
    assert knobs["trav_warps"] in (2, 4, 8) and knobs["enc_threads"] in (128, 256, 512)
    for poses in (poses_a, poses_b, poses_a):
        plan.run(poses)
        nif.nif_sync_status(h.h)
        ref = nif.nif_query(h.h, poses, rays, inst_offsets=inst)
        torch.cuda.synchronize()
        assert torch.equal(hits.view(torch.int32), ref.view(torch.int32))
    assert int((hits[:, 7].view(torch.int32) & 0xff).ne(0).sum()) > 100
    plan.close()
    h.close()


# ---------------------------------------------------------------------------
# Checkpoint / resume
# ---------------------------------------------------------------------------
def test_checkpoint_roundtrip_and_resume(nif, torus):
    import zlib
    net = S.NetConfig(levels=8, log2_table=12)
    a = nif.Nif(net, torus, seed=3)
    for step in range(5):
        nif.nif_train_step(a.h, 1 << 13, 4, 100 + step, want_loss=False)
    blob = nif.nif_checkpoint_save(a.h)
    # format: header magic, CRC-32 (IEEE, as zlib computes it) of everything before the trailer
    assert blob[:8] == b"NIFCKPT1"
    assert int.from_bytes(blob[-4:], "little") == zlib.crc32(blob[:-4])
    b = nif.Nif(net, torus, seed=99)
    nif.nif_checkpoint_load(b.h, blob)
    assert nif.nif_checkpoint_save(b.h) == blob               # state restored exactly
    la, _ = nif.nif_train_step(a.h, 1 << 13, 4, 777)
    lb, _ = nif.nif_train_step(b.h, 1 << 13, 4, 777)
    np.testing.assert_allclose(la, lb, rtol=1e-6)              # same batch, same state, same loss
    ta, wa, sa = a.get_params()
    tb, wb, sb = b.get_params()
    # gradients are summed with float atomics (order varies), so the updated state
    # agrees up to rounding; an entry whose tiny gradient flips sign on its first
    # Adam step moves by 2 lr, which only a handful of entries may do
    assert np.mean(np.abs(tb - ta) > 1e-6) < 1e-3
    for x, y in zip(wa, wb):
        np.testing.assert_allclose(y, x, atol=1e-5)
    bad = bytearray(blob)
    bad[100] ^= 1
    with pytest.raises(nif.NifError) as e:
        nif.nif_checkpoint_load(b.h, bytes(bad))
    assert e.value.status == nif.NIF_ERR_ARG
    other = nif.Nif(S.NetConfig(levels=4, log2_table=12), torus)
    with pytest.raises(nif.NifError):
        nif.nif_checkpoint_load(other.h, blob)
    for x in (a, b, other):
        x.close()
