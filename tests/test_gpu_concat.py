"""The concatenation reading of Eq. 1 (psi = [gamma, phi], NIF_FLAG_CONCAT_ENCODING)
through the C ABI against the FP64 oracle, and trained beside the default
reading psi = phi o gamma on the same data."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2604_24666_gb300 import synth as S
from tests.gpu_common import certain_rays, evaluate_hits, random_tables

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


def _lin(n, seed):
    """Linearized segments with end points around and slightly outside the cube."""
    rng = np.random.default_rng(seed)
    lin = np.zeros((n, 8), np.float32)
    lin[:, 0:3] = rng.uniform(-0.05, 1.05, (n, 3))
    lin[:, 3:6] = lin[:, 0:3] + rng.normal(0, 0.03, (n, 3))
    lin[:, 6] = lin[:, 7] = 1.0
    return lin


@pytest.mark.parametrize("levels,log2T", [(8, 14), (16, 19)])
def test_concat_forward_matches_oracle(nif, torus, levels, log2T):
    net = S.NetConfig(levels=levels, log2_table=log2T, encoding="concat")
    h = nif.Nif(net, torus)
    assert net.in_dim % 16 == 0 and net.in_dim >= 2 * net.point_width
    tables = random_tables(net, 171)
    h.set_params(tables, S.init_params(net)[1])
    lin = _lin(3001, 172)
    lt = torch.from_numpy(lin).to(_dev())
    p0, p1 = lin[:, 0:3].astype(np.float64), lin[:, 3:6].astype(np.float64)
    ref = O.encode_segments(net, tables, p0, p1)
    f = nif.nif_encode_segments(h.h, lt, net.in_dim).cpu().numpy()
    # gamma: sinf/cosf of an exact FP32 product (a few ulps); phi: the same FP32 cell decisions,
    # FP32 trilinear sums of 8 corners (|table| <= 1)
    np.testing.assert_allclose(f, ref, atol=2e-6, rtol=0)
    assert not f[:, 2 * net.point_width:].any()
    # 16-bit rows from the FP16 table copy: the oracle on FP16-rounded tables, BF16 rounding of the result
    t16 = tables.astype(np.float16).astype(np.float64)
    ref16 = O.encode_segments(net, t16, p0, p1)
    fb = nif.nif_encode_segments(h.h, lt, net.in_dim, out_dtype=nif.NIF_BF16, table_dtype=nif.NIF_FP16)
    fb = fb.float().cpu().numpy()
    np.testing.assert_allclose(fb, ref16, atol=1e-5, rtol=2.0 ** -8)
    h.close()


def test_concat_table_gradient_matches_oracle(nif, torus):
    net = S.NetConfig(levels=8, log2_table=12, encoding="concat")
    h = nif.Nif(net, torus)
    tables = random_tables(net, 173)
    h.set_params(tables, S.init_params(net)[1])
    lin = _lin(2500, 174)
    rng = np.random.default_rng(175)
    df = rng.normal(size=(len(lin), net.in_dim)).astype(np.float32)
    dtab = torch.zeros((net.levels, 1 << net.log2_table, 2), dtype=torch.float32, device=_dev())
    nif.nif_encode_segments_backward(h.h, torch.from_numpy(lin).to(_dev()), torch.from_numpy(df).to(_dev()), dtab)
    torch.cuda.synchronize()
    W = net.point_width
    r0, _ = O.encode_points_concat_backward(net, tables, lin[:, 0:3].astype(np.float64), df[:, :W].astype(np.float64))
    r1, _ = O.encode_points_concat_backward(net, tables, lin[:, 3:6].astype(np.float64),
                                            df[:, W:2 * W].astype(np.float64))
    ref = r0 + r1
    g = dtab.cpu().numpy()
    assert np.linalg.norm(g - ref) <= 1e-5 * np.linalg.norm(ref)
    h.close()


def test_concat_pose_gradient_matches_oracle(nif, torus):
    net = S.NetConfig(levels=8, log2_table=12, encoding="concat")
    N = net.voxel_res
    poses = np.array([[0.5, -0.9, 0.4], [-0.7, 0.6, -0.3]], np.float32)
    parts = []
    for i, seed in enumerate((176, 177)):
        r = S.sphere_rays(700, seed=seed)
        parts.append(r[certain_rays(N, torus, poses[i], r)])
    rays_np = np.concatenate(parts)
    inst = np.array([0, len(parts[0]), len(rays_np)], np.int32)
    h = nif.Nif(net, torus)
    tables = random_tables(net, 178, scale=0.5)
    h.set_params(tables, S.init_params(net)[1])
    rays = torch.from_numpy(rays_np).to(_dev())
    it = torch.from_numpy(inst).to(_dev())
    offs, segs = nif.nif_segments(h.h, poses, rays, inst_offsets=it)
    lin = nif.nif_linearize(h.h, poses, rays, segs, inst_offsets=it)
    n = segs.shape[0]
    df = np.random.default_rng(179).normal(size=(n, net.in_dim)).astype(np.float32)
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


def _mean(ds):
    return {k: float(np.mean([d[k] for d in ds])) for k in ds[0]}


def test_concat_reading_trains_beside_composed(nif, torus):
    """Both readings of Eq. 1 trained from the same seed on the 16^3 torus (4000
    FP32 steps of 2^16 segments, poses U[-1,1]^3), evaluated on held-out poses
    against the exact deformed-mesh hits. The concatenation must learn (beat
    its untrained network on hit IoU and distance); the two are reported side
    by side."""
    m = {}
    for enc in ("composed", "concat"):
        net = S.NetConfig(encoding=enc)
        trained = nif.Nif(net, torus, seed=7)
        init = nif.Nif(net, torus, seed=7)
        for step in range(4000):
            nif.nif_train_step(trained.h, 1 << 16, 16, 1000 + step, lr_grid=1e-2, lr_mlp=5e-3, want_loss=False)
        rays_np = S.sphere_rays(2500, seed=4343)
        rays = torch.from_numpy(rays_np).to(_dev())
        for name, hh in (("trained", trained), ("init", init)):
            ds = []
            for pose in S.poses(4, seed=4242):
                hq = nif.nif_query(hh.h, [pose], rays).cpu().numpy().view(nif.HIT_DTYPE).reshape(-1)
                ds.append(evaluate_hits(torus, pose, rays_np, hq["hit"] > 0, hq["D"].astype(np.float64),
                                        hq["n"].astype(np.float64), hq["albedo"], hq["material"]))
            m[(enc, name)] = _mean(ds)
        trained.close()
        init.close()
    print("readings of Eq. 1:", {f"{e}/{n}": v for (e, n), v in m.items()})
    c, ci = m[("concat", "trained")], m[("concat", "init")]
    assert c["iou"] > ci["iou"] and c["iou"] > 0.9
    assert c["dist"] < ci["dist"]
    assert m[("composed", "trained")]["iou"] > 0.95
