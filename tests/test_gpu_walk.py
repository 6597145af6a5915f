"""Segments by the paper's traversal (Sec. 2.1: BVH first hit, then a walk
through the exit faces of the deformed voxels, a new BVH query after leaving
the grid), through the C ABI, against the FP64 oracle's segment definition and
against the library's enumeration of every occupied hull."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2604_24666_gb300 import synth as S
from tests.gpu_common import SEG_MARGIN

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


def _rows(offs, segs, nif):
    return offs.cpu().numpy().astype(np.int64), segs.cpu().numpy().view(nif.SEGMENT_DTYPE).reshape(-1)


@pytest.mark.parametrize("shape,N,pose,n_rays", [
    ("torus", 16, (0.0, 0.0, 0.0), 2000),
    ("torus", 16, (0.4, -0.7, 0.3), 2000),
    ("torus", 16, (1.0, -1.5, 1.0), 2000),
    ("ellipsoids", 32, (-1.0, 1.0, -1.0), 1500),
    ("ellipsoids", 64, (0.6, 0.9, -0.5), 600),
])
def test_walk_matches_oracle_and_enumeration(nif, torus, ellipsoids, shape, N, pose, n_rays):
    mesh = torus if shape == "torus" else ellipsoids
    rays_np = S.sphere_rays(n_rays, seed=41)
    h = nif.Nif(S.NetConfig(voxel_res=N), mesh)
    rays = torch.from_numpy(rays_np).to(_dev())
    ow, gw = _rows(*nif.nif_segments_walk(h.h, [pose], rays), nif)
    oe, ge = _rows(*nif.nif_segments(h.h, [pose], rays), nif)
    occ, _, _ = O.voxelize(N, mesh)
    seg = O.segments(N, occ, pose, rays_np)
    certain = seg.margin > SEG_MARGIN
    assert certain.mean() > 0.8
    for r in np.nonzero(certain)[0]:
        w = gw[ow[r]:ow[r + 1]]
        assert np.array_equal(w["voxel"], seg.vox[seg.off[r]:seg.off[r + 1]]), r
        # the same hull test on the same corners: the enumeration's row, field for field
        assert np.array_equal(w, ge[oe[r]:oe[r + 1]]), r
    # every row is sorted by t0; rays decided with less margin still agree almost always
    same = 0
    for r in range(n_rays):
        w = gw[ow[r]:ow[r + 1]]
        assert np.all(np.diff(w["t0"]) >= 0)
        same += np.array_equal(w, ge[oe[r]:oe[r + 1]])
    assert same >= 0.995 * n_rays, same
    # the first BVH query alone finds a hull exactly on the rays that have segments
    fo, none = nif.nif_segments_walk(h.h, [pose], rays, flags=nif.NIF_WALK_FIRST_HIT)
    assert none is None
    assert int(fo[-1].item()) == int((np.diff(oe) > 0).sum())
    h.close()


def test_walk_multi_instance(nif, torus):
    N = 16
    poses = S.poses(4, seed=43)
    counts = [300, 0, 900, 450]
    rays_np = S.sphere_rays(sum(counts), seed=44)
    inst = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    inst_dev = torch.from_numpy(inst).to(_dev())
    h = nif.Nif(S.NetConfig(voxel_res=N), torus)
    rays = torch.from_numpy(rays_np).to(_dev())
    ow, gw = _rows(*nif.nif_segments_walk(h.h, poses, rays, inst_offsets=inst_dev), nif)
    oe, ge = _rows(*nif.nif_segments(h.h, poses, rays, inst_offsets=inst_dev), nif)
    occ, _, _ = O.voxelize(N, torus)
    n_cmp = 0
    for i in range(len(counts)):
        sub = rays_np[inst[i]:inst[i + 1]]
        if not len(sub):
            continue
        seg = O.segments(N, occ, poses[i], sub)
        for r in np.nonzero(seg.margin > SEG_MARGIN)[0]:
            R = inst[i] + r
            assert np.array_equal(gw["voxel"][ow[R]:ow[R + 1]], seg.vox[seg.off[r]:seg.off[r + 1]]), R
            assert np.array_equal(gw[ow[R]:ow[R + 1]], ge[oe[R]:oe[R + 1]]), R
            n_cmp += 1
    assert n_cmp > 1400
    h.close()


def test_walk_rejects_bad_arguments(nif, torus):
    h = nif.Nif(S.NetConfig(voxel_res=16), torus)
    rays = torch.from_numpy(S.sphere_rays(64, seed=45)).to(_dev())
    offs = torch.zeros(65, dtype=torch.int32, device=_dev())
    segs = torch.zeros((16, 4), dtype=torch.int32, device=_dev())
    pose = (nif.nif_pose * 1)(nif.nif_pose(0.0, 0.0, 0.0))
    total = nif._i64()
    lib = nif.lib()
    # the first-hit mode counts only; an unknown flag is refused
    assert lib.nif_segments_walk(h.h, pose, 1, nif._ptr(rays), None, 64, nif._ptr(offs), nif._ptr(segs), 16,
                                 nif.ctypes.byref(total), nif.NIF_WALK_FIRST_HIT, None) == nif.NIF_ERR_ARG
    assert lib.nif_segments_walk(h.h, pose, 1, nif._ptr(rays), None, 64, nif._ptr(offs), None, 0,
                                 nif.ctypes.byref(total), 2, None) == nif.NIF_ERR_ARG
    h.close()
