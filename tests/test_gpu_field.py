"""The learned deformation field on the GPU (our reading of the paper's Sec. 4
future work: per instance a trilinear lattice of rest-space displacements
composed before the parameterised deformation, D(p) = D_pose(p + u(p))),
against the FP64 oracle's `deform_field` family on the same inputs:
segments (bit-exact voxel sequences on rays decided with margin), the
Newton inverse of the linearization, the query's hits and normals, the
gradient with respect to the field and the pose gradient under a field. A
fitting test shows the field moving towards a target deformation from
intersection supervision alone.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2604_24666_gb300 import synth as S
from tests import bounds as B
from tests.gpu_common import SEG_MARGIN, occupancy_biased_weights, random_tables

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


def _dev():
    return torch.device("cuda:0")


def _field(G, seed, lip=0.4):
    f = np.random.default_rng(seed).normal(size=(G, G, G, 3))
    return (f * (lip / O.field_lipschitz(f))).astype(np.float32)


@pytest.mark.parametrize("pose", [(0.0, 0.0, 0.0), (0.6, -0.9, 0.4)])
def test_field_segments_and_linearization_match_oracle(nif, torus, pose):
    N = 16
    f = _field(5, 401)
    h = nif.Nif(S.NetConfig(voxel_res=N), torus)
    nif.nif_set_field(h.h, f[None])
    got = nif.nif_get_field(h.h)
    assert np.array_equal(got[0], f)
    rays_np = S.sphere_rays(2500, seed=402)
    rays = torch.from_numpy(rays_np).to(_dev())
    offs, segs = nif.nif_segments(h.h, [pose], rays)
    off = offs.cpu().numpy().astype(np.int64)
    g = segs.cpu().numpy().view(nif.SEGMENT_DTYPE).reshape(-1)
    occ, _, _ = O.voxelize(N, torus)
    f64 = f.astype(np.float64)
    seg = O.segments(N, occ, pose, rays_np, field=f64)
    certain = seg.margin > SEG_MARGIN
    assert certain.mean() > 0.95
    dt = []
    for r in np.nonzero(certain)[0]:
        gv = g[off[r]:off[r + 1]]
        a, b = seg.off[r], seg.off[r + 1]
        assert np.array_equal(gv["voxel"], seg.vox[a:b]), r
        dt.append(np.abs(gv["t0"] - seg.t0[a:b]))
        dt.append(np.abs(gv["t1"] - seg.t1[a:b]))
    dt = np.concatenate(dt)
    assert np.median(dt) < 1e-6 and dt.max() < 1e-3, (np.median(dt), dt.max())
    # linearization on the rays decided with margin (same segment lists)
    keep = np.nonzero(certain)[0]
    rk = torch.from_numpy(rays_np[keep]).to(_dev())
    _, sk = nif.nif_segments(h.h, [pose], rk)
    lin = nif.nif_linearize(h.h, [pose], rk, sk).cpu().numpy().view(nif.LINSEG_DTYPE).reshape(-1)
    sref = O.segments(N, occ, pose, rays_np[keep], field=f64)
    p0, p1, ld, lr = O.linearize(pose, rays_np[keep], sref, field=f64)
    assert len(lin) == len(sref)
    # t error times |dD^-1/dx| (the field's bound 0.4 adds a factor 1/(1 - 0.4)), plus the FP32 Newton residual
    np.testing.assert_allclose(lin["p0"], p0, atol=5e-4)
    np.testing.assert_allclose(lin["p1"], p1, atol=5e-4)
    assert np.median(np.abs(lin["p0"] - p0)) < 4e-6
    np.testing.assert_allclose(lin["l_rest"], lr, atol=1e-3)
    h.close()


def test_field_query_matches_oracle(nif, torus):
    net = S.NetConfig()
    pose = (0.4, -0.7, 0.3)
    f = _field(5, 411, lip=0.3)
    f64 = f.astype(np.float64)
    h = nif.Nif(net, torus)
    tables = random_tables(net, 412)
    ws, s = occupancy_biased_weights(net, 413)
    h.set_params(tables, ws, s)
    nif.nif_set_field(h.h, f[None])
    rays_np = S.sphere_rays(1500, seed=414)
    occ, _, _ = O.voxelize(net.voxel_res, torus)
    seg = O.segments(net.voxel_res, occ, pose, rays_np, field=f64)
    rays_np = rays_np[seg.margin > SEG_MARGIN]
    hits = nif.nif_query(h.h, [pose], torch.from_numpy(rays_np).to(_dev())).cpu().numpy()
    hits = hits.view(nif.HIT_DTYPE).reshape(-1)
    seg = O.segments(net.voxel_res, occ, pose, rays_np, field=f64)
    p0, p1, ld, lr = O.linearize(pose, rays_np, seg, field=f64)
    out = O.mlp_forward(ws, O.encode_segments(net, tables, p0, p1))[0]
    res = O.reconstruct(net, pose, rays_np, seg, out, p0, p1, ld, lr, field=f64)
    n_cmp = 0
    for r in range(len(rays_np)):
        a, b = seg.off[r], seg.off[r + 1]
        if np.any(np.abs(out[a:b, 0]) < 1e-3):
            continue
        assert hits["hit"][r] == res["hit"][r], r
        if res["hit"][r]:
            assert abs(hits["D"][r] - res["D"][r]) < 5e-4, (r, hits["D"][r], res["D"][r])
            assert np.dot(hits["n"][r], res["normal"][r]) > np.cos(np.radians(0.1))
        n_cmp += 1
    assert n_cmp > 700 and hits["hit"].sum() > 100
    h.close()


def test_field_gradient_matches_oracle(nif, torus):
    """Element by element on identical inputs: linearized segments from the
    generator (cells certain), random feature gradients. Node bound: the
    end points' dL/dp bounds (tests/bounds.py) carried through
    |(I + du/dp)^-T| <= 1/(1 - 0.4) (the field's bound) and the trilinear weights, plus FP32
    rounding of the solve and of the atomic sums."""
    net = S.NetConfig(levels=8, log2_table=12)
    G = 5
    f = _field(G, 421, lip=0.4)
    f64 = f.astype(np.float64)
    pose = (0.3, -0.5, 0.2)
    h = nif.Nif(net, torus)
    tables = random_tables(net, 422, scale=0.5)
    h.set_params(tables, S.init_params(net)[1])
    nif.nif_set_field(h.h, f[None])
    lin, _ = S.chained_segments(4000, seed=423, voxel_res=16, gap=0.2, margin=0.0)
    ok = B.certain_cells(net, lin[:, 0:3]) & B.certain_cells(net, lin[:, 3:6])
    lin = lin[ok][:2000]
    n = len(lin)
    segs = np.zeros((n, 4), np.int32)            # one instance: ray 0 for every segment
    df = np.random.default_rng(424).normal(size=(n, net.in_dim)).astype(np.float32)
    got = nif.nif_field_gradient(h.h, [pose], torch.from_numpy(segs).to(_dev()), torch.from_numpy(lin).to(_dev()),
                                 torch.from_numpy(df).to(_dev())).cpu().numpy()[0]
    p0, p1 = lin[:, 0:3].astype(np.float64), lin[:, 3:6].astype(np.float64)
    ref = O.field_gradient(net, tables, pose, f64, p0, p1, df.astype(np.float64))
    half = net.in_dim // 2
    bound = np.zeros_like(ref)
    cnt = np.zeros(ref.shape[:3])
    for p, d in ((p0, df[:, :half].astype(np.float64)), (p1, df[:, half:].astype(np.float64))):
        bdp = B.point_grad_bound(net, tables, p, d).sum(1)
        _, dp = O.encode_points_backward(net, tables, p, d)
        A = np.eye(3)[None] + O.field_grad(f64, p)
        v = np.linalg.solve(np.transpose(A, (0, 2, 1)), dp[..., None])[..., 0]
        i0, t, _ = O.field_cell(f64, p)
        for c in O._CORNERS:
            w = np.prod(np.where(c == 1, t, 1.0 - t), axis=1)
            nn = i0 + c
            e = w[:, None] * (bdp[:, None] / (1 - 0.4) + 1e-6 * np.abs(v).sum(1, keepdims=True) + 8 * B.U32 * np.abs(v))
            np.add.at(bound, (nn[:, 2], nn[:, 1], nn[:, 0]), e)
            np.add.at(cnt, (nn[:, 2], nn[:, 1], nn[:, 0]), 1.0)
    absum = np.zeros_like(ref)
    for p, d in ((p0, df[:, :half]), (p1, df[:, half:])):
        _, dp = O.encode_points_backward(net, tables, p, d.astype(np.float64))
        A = np.eye(3)[None] + O.field_grad(f64, p)
        v = np.abs(np.linalg.solve(np.transpose(A, (0, 2, 1)), dp[..., None])[..., 0])
        i0, t, _ = O.field_cell(f64, p)
        for c in O._CORNERS:
            w = np.prod(np.where(c == 1, t, 1.0 - t), axis=1)
            nn = i0 + c
            np.add.at(absum, (nn[:, 2], nn[:, 1], nn[:, 0]), w[:, None] * v)
    bound += (cnt[..., None] + 4) * B.U32 * absum
    err = np.abs(got - ref)
    assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).max()
    assert np.abs(ref).max() > 0
    h.close()


@pytest.mark.parametrize("bands", [0, 4])
def test_pose_gradient_under_a_field_matches_oracle(nif, torus, bands):
    """d/d(bend, twist, taper) with a field under the pose, on identical rest
    points (generated, cells certain) and feature gradients. Bound: each end
    point's dL/dp bound (tests/bounds.py) carried through |dp/dtheta| =
    |(I + du/dp)^-1 J_pose(q)^-1 dD_pose/dtheta(q)|, plus 1e-5 of the sum of
    the absolute terms for the FP32 Jacobians and solves. Without the
    positional bands the bound is rounding only (about 1e-3 of the result);
    with them it carries the sincosf allowance of every sin/cos cell."""
    net = S.NetConfig(levels=8, log2_table=12, pe_bands=bands)
    f = _field(4, 431, lip=0.35)
    f64 = f.astype(np.float64)
    pose = np.array([[0.5, -0.9, 0.4]], np.float32)
    h = nif.Nif(net, torus)
    tables = random_tables(net, 433, scale=0.5)
    h.set_params(tables, S.init_params(net)[1])
    nif.nif_set_field(h.h, f[None])
    lin, _ = S.chained_segments(3000, seed=435, voxel_res=16, gap=0.2, margin=0.0)
    ok = B.certain_cells(net, lin[:, 0:3]) & B.certain_cells(net, lin[:, 3:6])
    lin = lin[ok][:1500]
    n = len(lin)
    segs = np.zeros((n, 4), np.int32)                # one instance
    df = np.random.default_rng(434).normal(size=(n, net.in_dim)).astype(np.float32)
    dposes = nif.nif_pose_gradient(h.h, pose, torch.from_numpy(segs).to(_dev()), torch.from_numpy(lin).to(_dev()),
                                   torch.from_numpy(df).to(_dev()))
    got = dposes.cpu().numpy()[0]
    p0, p1 = lin[:, 0:3].astype(np.float64), lin[:, 3:6].astype(np.float64)
    ref = O.pose_gradient(net, tables, pose[0], p0, p1, df.astype(np.float64), field=f64)
    half = net.in_dim // 2
    bound = np.zeros(3)
    for p, d in ((p0, df[:, :half].astype(np.float64)), (p1, df[:, half:].astype(np.float64))):
        _, dp = O.encode_points_backward(net, tables, p, d)
        q = p + O.field_displacement(f64, p)
        J, Jp = O.jacobians(pose[0], q)
        A = -np.linalg.solve(np.eye(3)[None] + O.field_grad(f64, p), np.linalg.solve(J, Jp))   # dp/dtheta
        bd = B.point_grad_bound(net, tables, p, d)
        bound += np.einsum("na,naj->j", bd, np.abs(A)) + 1e-5 * np.einsum("na,naj->j", np.abs(dp), np.abs(A))
    assert np.all(np.abs(got - ref) <= bound), (got, ref, bound)
    h.close()


def test_field_checks(nif, torus):
    h = nif.Nif(S.NetConfig(), torus)
    bad = _field(4, 441, lip=0.95)                 # Lipschitz bound above 0.9
    with pytest.raises(nif.NifError) as e:
        nif.nif_set_field(h.h, bad[None])
    assert e.value.status == nif.NIF_ERR_ARG
    nif.nif_set_field(h.h, _field(4, 442)[None])
    rays = torch.from_numpy(S.sphere_rays(64, seed=443)).to(_dev())
    inst = torch.tensor([0, 32, 64], dtype=torch.int32, device=_dev())
    with pytest.raises(nif.NifError) as e:           # two instances, one field
        nif.nif_query(h.h, [(0, 0, 0), (0, 0, 0)], rays, inst_offsets=inst)
    assert e.value.status == nif.NIF_ERR_ARG
    nif.nif_set_field(h.h, None)
    assert nif.nif_get_field(h.h) is None
    nif.nif_query(h.h, [(0, 0, 0), (0, 0, 0)], rays, inst_offsets=inst)
    h.close()


def test_field_fitting_moves_towards_the_target(nif, torus):
    """A network trained over random poses knows the rest shape. The
    deformation of an instance is known only in part (its pose is half the
    target twist); a field fitted under that pose by nif_field_step, to
    labels taken along the rest segments of the target twist, must move the
    deformed mesh towards the target's: the mean distance between D(v) and
    D_target(v) over the mesh vertices falls well below its value for the
    zero field."""
    net = S.NetConfig()
    h = nif.Nif(net, torus, seed=7)
    for step in range(1500):
        nif.nif_train_step(h.h, 1 << 14, 8, 9000 + step, lr_grid=1e-2, lr_mlp=5e-3, want_loss=False)
    G = 5
    nif.nif_set_field(h.h, np.zeros((1, G, G, G, 3), np.float32))
    target = np.array([[0.0, 1.4, 0.0]], np.float32)
    pose = np.array([[0.0, 0.7, 0.0]], np.float32)
    verts = torus.verts.astype(np.float64)
    goal = O.deform(target[0], verts)

    def mesh_error():
        f = nif.nif_get_field(h.h)[0].astype(np.float64)
        return float(np.linalg.norm(O.deform_field(pose[0], f, verts) - goal, axis=1).mean())

    e0 = mesh_error()
    losses = []
    for step in range(600):
        rays = torch.from_numpy(S.sphere_rays(6000, seed=10000 + step)).to(_dev())
        loss = nif.nif_field_step(h.h, pose, rays, 1 << 14, target, lr_field=2e-3, want_loss=(step % 50 == 0))
        if loss is not None:
            losses.append(loss[0])
    e1 = mesh_error()
    assert e1 < 0.5 * e0, (e0, e1, losses)
    assert losses[-1] < losses[0]
    f = nif.nif_get_field(h.h)[0].astype(np.float64)
    assert O.field_lipschitz(f) <= 0.9 + 1e-5
    h.close()


def test_checkpoint_carries_the_field(nif, torus):
    """A checkpoint holds the learned field (displacements, Adam moments and
    step count): loaded into a fresh handle it gives the same field and
    saves to the same bytes, and the next field step of both handles moves
    the field alike; a checkpoint taken without a field removes one."""
    net = S.NetConfig()
    a = nif.Nif(net, torus, seed=7)
    bare = nif.nif_checkpoint_save(a.h)
    nif.nif_set_field(a.h, _field(5, 451, lip=0.2)[None])
    pose = np.array([[0.0, 0.7, 0.0]], np.float32)
    target = np.array([[0.0, 1.0, 0.0]], np.float32)
    for step in range(3):
        rays = torch.from_numpy(S.sphere_rays(6000, seed=452 + step)).to(_dev())
        nif.nif_field_step(a.h, pose, rays, 1 << 13, target, lr_field=2e-3, want_loss=False)
    blob = nif.nif_checkpoint_save(a.h)
    assert len(blob) == len(bare) + 3 * 16 * 5 ** 3
    b = nif.Nif(net, torus, seed=99)
    nif.nif_checkpoint_load(b.h, blob)
    assert nif.nif_checkpoint_save(b.h) == blob
    assert np.array_equal(nif.nif_get_field(b.h), nif.nif_get_field(a.h))
    rays = torch.from_numpy(S.sphere_rays(6000, seed=460)).to(_dev())
    for x in (a, b):
        nif.nif_field_step(x.h, pose, rays, 1 << 13, target, lr_field=2e-3, want_loss=False)
    # field gradients are summed with float atomics: the same step to rounding
    np.testing.assert_allclose(nif.nif_get_field(b.h), nif.nif_get_field(a.h), atol=1e-6)
    nif.nif_checkpoint_load(b.h, bare)
    assert nif.nif_get_field(b.h) is None
    for x in (a, b):
        x.close()
