"""The curved-face reading of a deformed voxel (NIF_FLAG_BILINEAR_FACES: each
face the bilinear patch of its four deformed corners) through the C ABI
against the FP64 oracle's segments, and trained end to end."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2604_24666_gb300 import synth as S
from tests.gpu_common import SEG_MARGIN, evaluate_hits

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


def _segments(nif, h, poses, rays_np, inst=None):
    rays = torch.from_numpy(rays_np).to(_dev())
    it = None if inst is None else torch.from_numpy(inst).to(_dev())
    offs, segs = nif.nif_segments(h.h, poses, rays, inst_offsets=it)
    return offs.cpu().numpy().astype(np.int64), segs.cpu().numpy().view(nif.SEGMENT_DTYPE).reshape(-1)


@pytest.mark.parametrize("pose", [(0, 0, 0), (0.4, -0.7, 0.3), (-1.0, 1.0, -1.0), (1.0, -1.5, 1.0)])
def test_bilinear_segments_match_oracle(nif, torus, pose):
    """Voxel sequences bit-exact on rays the oracle decides with margin (its
    margin also counts the distance to every face edge of the hulls the ray
    meets: the FP32 patch test is not watertight there)."""
    N = 16
    rays_np = S.sphere_rays(3000, seed=21)
    h = nif.Nif(S.NetConfig(voxel_res=N, faces="bilinear"), torus)
    off, g = _segments(nif, h, [pose], rays_np)
    occ, _, _ = O.voxelize(N, torus)
    seg = O.segments(N, occ, pose, rays_np, faces="bilinear")
    certain = seg.margin > SEG_MARGIN
    assert certain.mean() > 0.97
    dt = []
    for r in np.nonzero(certain)[0]:
        gv = g[off[r]:off[r + 1]]
        a, b = seg.off[r], seg.off[r + 1]
        assert np.array_equal(gv["voxel"], seg.vox[a:b]), r
        dt.append(np.abs(gv["t0"] - seg.t0[a:b]))
        dt.append(np.abs(gv["t1"] - seg.t1[a:b]))
    dt = np.concatenate(dt)
    # FP32 corners (~5e-7) through the quadratic's conditioning; grazing hits make the tail
    assert np.median(dt) < 2e-6 and dt.max() < 2e-3, (np.median(dt), np.percentile(dt, 99), dt.max())
    for r in range(len(rays_np)):
        assert np.all(np.diff(g[off[r]:off[r + 1]]["t0"]) >= 0)
    h.close()


def test_bilinear_multi_instance_and_ellipsoids64(nif, torus):
    N = 16
    poses = S.poses(3, seed=41)
    counts = [700, 0, 900]
    rays_np = S.sphere_rays(sum(counts), seed=42)
    inst = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    h = nif.Nif(S.NetConfig(voxel_res=N, faces="bilinear"), torus)
    off, g = _segments(nif, h, poses, rays_np, inst)
    occ, _, _ = O.voxelize(N, torus)
    n_cmp = 0
    for i in range(3):
        sub = rays_np[inst[i]:inst[i + 1]]
        if not len(sub):
            continue
        seg = O.segments(N, occ, poses[i], sub, faces="bilinear")
        for r in np.nonzero(seg.margin > SEG_MARGIN)[0]:
            R = inst[i] + r
            assert np.array_equal(g["voxel"][off[R]:off[R + 1]], seg.vox[seg.off[r]:seg.off[r + 1]])
            n_cmp += 1
    assert n_cmp > 1000
    h.close()
    ell = S.ellipsoid_union_mesh()
    N = 64
    pose = (0.6, 0.9, -0.5)
    rays_np = S.sphere_rays(400, seed=43)
    h = nif.Nif(S.NetConfig(voxel_res=N, faces="bilinear"), ell)
    off, g = _segments(nif, h, [pose], rays_np)
    occ, _, _ = O.voxelize(N, ell)
    seg = O.segments(N, occ, pose, rays_np, faces="bilinear")
    certain = seg.margin > SEG_MARGIN
    assert certain.mean() > 0.8
    for r in np.nonzero(certain)[0]:
        assert np.array_equal(g["voxel"][off[r]:off[r + 1]], seg.vox[seg.off[r]:seg.off[r + 1]]), r
    h.close()


def test_bilinear_planar_faces_equal_triangles(nif, torus):
    """At the identity pose the faces are planar squares: both readings give
    the same segments on the GPU too."""
    N = 16
    rays_np = S.sphere_rays(3000, seed=44)
    a = nif.Nif(S.NetConfig(voxel_res=N), torus)
    b = nif.Nif(S.NetConfig(voxel_res=N, faces="bilinear"), torus)
    oa, ga = _segments(nif, a, [(0.0, 0.0, 0.0)], rays_np)
    ob, gb = _segments(nif, b, [(0.0, 0.0, 0.0)], rays_np)
    occ, _, _ = O.voxelize(N, torus)
    seg = O.segments(N, occ, (0.0, 0.0, 0.0), rays_np, faces="bilinear")
    for r in np.nonzero(seg.margin > SEG_MARGIN)[0]:
        assert np.array_equal(ga["voxel"][oa[r]:oa[r + 1]], gb["voxel"][ob[r]:ob[r + 1]])
        np.testing.assert_allclose(gb["t0"][ob[r]:ob[r + 1]], ga["t0"][oa[r]:oa[r + 1]], atol=2e-6)
    a.close()
    b.close()


def test_walk_refuses_bilinear_faces(nif, torus):
    h = nif.Nif(S.NetConfig(faces="bilinear"), torus)
    rays = torch.from_numpy(S.sphere_rays(64, seed=45)).to(_dev())
    with pytest.raises(nif.NifError):
        nif.nif_segments_walk(h.h, [(0.1, 0.2, 0.3)], rays)
    h.close()


def test_bilinear_faces_train_and_query(nif, torus):
    """Trained with curved faces (3000 FP32 steps of 2^16 segments on the 16^3
    torus, poses U[-1,1]^3) and evaluated on held-out poses against the exact
    deformed-mesh hits: it must learn as the triangulated reading does."""
    net = S.NetConfig(faces="bilinear")
    trained = nif.Nif(net, torus, seed=7)
    for step in range(3000):
        nif.nif_train_step(trained.h, 1 << 16, 16, 1000 + step, lr_grid=1e-2, lr_mlp=5e-3, want_loss=False)
    loss, _ = nif.nif_train_step(trained.h, 1 << 16, 16, 99999, lr_grid=0.0, lr_mlp=0.0, want_loss=True)
    assert np.isfinite(loss).all()
    rays_np = S.sphere_rays(2500, seed=4343)
    rays = torch.from_numpy(rays_np).to(_dev())
    ious, dists = [], []
    for pose in S.poses(4, seed=4242):
        hq = nif.nif_query(trained.h, [pose], rays).cpu().numpy().view(nif.HIT_DTYPE).reshape(-1)
        m = evaluate_hits(torus, pose, rays_np, hq["hit"] > 0, hq["D"].astype(np.float64),
                          hq["n"].astype(np.float64), hq["albedo"], hq["material"])
        ious.append(m["iou"])
        dists.append(m["dist"])
    print("bilinear faces: hit IoU", np.mean(ious), "distance MAE", np.mean(dists))
    assert np.mean(ious) > 0.95 and np.mean(dists) < 0.03
    trained.close()
