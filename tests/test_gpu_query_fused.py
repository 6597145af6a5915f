"""The BF16/FP16 query with its encoding (Eq. 1) computed inside the
tensor-core MLP kernel (NIF_KNOB_QUERY_FUSED, the default): features of a
tile go from the producer warps into the MMA's shared-memory ring and never
reach global memory.

* Against the FP64 oracle for each level count, width and depth the kernel
  covers, on the same weights (hit agreement on rays whose occupancy logits
  are clear of 5 % of their range, distance <= 2e-3, albedo <= 2e-2, normal
  within 2 degrees on 99 % of the hits and 5 on all, material >= 99 % where
  the top two logits are clear), and against the two-kernel path on the
  same handle.
* Against the two-kernel path (NIF_KNOB_QUERY_FUSED = 0) at the 128^3
  query workload's full size (2^22 rays, ~19 M segments, one launch of the
  fused kernel over ~150 k tiles): the two differ in layer 0's
  accumulation order and in the sine and cosine of gamma (the fused kernel
  takes the fast intrinsics), so the hit decisions agree except where a
  logit is within rounding of zero.
* Edge cases: a query whose rays all miss the grid (no segment: the kernel
  launches with a zero device count), and ray counts that leave a ragged
  last tile.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2604_24666_gb300 import synth as S
from tests.gpu_common import certain_rays, occupancy_biased_weights, random_tables

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


def _check_against_oracle(nif, net, mesh, hits, tables, ws, pose, rays_np):
    """Rays whose occupancy logits are all clear of 5 % of their range: the
    hit decision equals the oracle's; on hits, distance <= 2e-3 and albedo
    <= 2e-2 everywhere; the normal within 2 degrees on 99 % of the rays and
    within 5 degrees on all where the raw normal vector is longer than 10 %
    of the longest (a short one turns further under the same 16-bit rounding
    of the outputs, as a logit near zero flips); material >= 99 % where the
    top two logits are clear."""
    occ, _, _ = O.voxelize(net.voxel_res, mesh)
    seg = O.segments(net.voxel_res, occ, pose, rays_np)
    p0, p1, ld, lr = O.linearize(pose, rays_np, seg)
    out = O.mlp_forward(ws, O.encode_segments(net, tables, p0, p1))[0]
    res = O.reconstruct(net, pose, rays_np, seg, out, p0, p1, ld, lr)
    zr = np.abs(out[:, 0]).max()
    nlen = np.linalg.norm(out[:, 2:5], axis=1)
    nmax = nlen.max()
    n_cmp, mat_ok, mat_n, ang = 0, 0, 0, []
    for r in range(len(rays_np)):
        a, b = seg.off[r], seg.off[r + 1]
        if np.any(np.abs(out[a:b, 0]) < 0.05 * zr):
            continue
        assert hits["hit"][r] == res["hit"][r], r
        if res["hit"][r]:
            j = a + res["k"][r]
            assert abs(hits["D"][r] - res["D"][r]) < 2e-3, (r, hits["D"][r], res["D"][r])
            np.testing.assert_allclose(hits["albedo"][r], res["albedo"][r], atol=2e-2)
            if nlen[j] > 0.1 * nmax:
                ang.append(np.degrees(np.arccos(np.clip(np.dot(hits["n"][r], res["normal"][r]), -1.0, 1.0))))
            m = np.sort(out[j, 8:12])
            if m[-1] - m[-2] > 0.05 * (np.abs(out[:, 8:12]).max()):
                mat_n += 1
                mat_ok += hits["material"][r] == res["material"][r]
        n_cmp += 1
    ang = np.asarray(ang)
    if ang.size:
        assert np.percentile(ang, 99) <= 2.0 and ang.max() <= 5.0, (np.percentile(ang, 99), ang.max())
    assert mat_n == 0 or mat_ok >= 0.99 * mat_n
    return n_cmp, ang.size


@pytest.mark.parametrize("levels,log2T,width,depth", [(8, 14, 32, 2), (16, 14, 64, 3), (4, 12, 32, 1), (16, 13, 32, 2),
                                                      (8, 15, 64, 3), (8, 14, 64, 4)])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_fused_query_matches_oracle(nif, torus, levels, log2T, width, depth, prec):
    """The fused query against the oracle, and against the two-kernel path on
    the same handle: 16-bit features that differ by the fast sine's error at
    most, layer 0 summed in another order, so the two agree to the rounding
    of an activation."""
    net = S.NetConfig(levels=levels, log2_table=log2T, mlp_depth=depth, mlp_width=width)
    p = nif.NIF_BF16 if prec == "bf16" else nif.NIF_FP16
    h = nif.Nif(net, torus, precision=p)
    tables = random_tables(net, 301 + levels)
    ws, s = occupancy_biased_weights(net, 302 + width)
    h.set_params(tables, ws, s)
    pose = (-0.4, 0.9, 0.3)
    rays_np = S.sphere_rays(2000 + 77, seed=303)         # ragged last tile of segments
    rays_np = rays_np[certain_rays(net.voxel_res, torus, pose, rays_np)]
    rays = torch.from_numpy(rays_np).to(_dev())
    nif.nif_set_knob(h.h, nif.NIF_KNOB_QUERY_FUSED, 1)
    hits = nif.nif_query(h.h, [pose], rays).cpu().numpy().view(nif.HIT_DTYPE).reshape(-1)
    nif.nif_set_knob(h.h, nif.NIF_KNOB_QUERY_FUSED, 0)
    two = nif.nif_query(h.h, [pose], rays).cpu().numpy().view(nif.HIT_DTYPE).reshape(-1)
    nif.nif_sync_status(h.h)
    h.close()
    n_cmp, n_hit = _check_against_oracle(nif, net, torus, hits, tables, ws, pose, rays_np)
    assert n_cmp > 500 and n_hit > 50
    both = (hits["hit"] > 0) & (two["hit"] > 0)
    assert both.sum() >= 0.99 * ((hits["hit"] > 0) | (two["hit"] > 0)).sum()
    same = both.copy()
    same[both] = np.abs(hits["D"][both] - two["D"][both]) < 2e-3
    assert same.sum() >= 0.99 * both.sum()
    assert np.abs(hits["D"][same] - two["D"][same]).max() < 1e-3
    cosang = (hits["n"][same] * two["n"][same]).sum(1)
    assert np.percentile(cosang, 1) > np.cos(np.radians(1.0))


def test_fused_query_full_size_matches_two_kernel_path(nif):
    """2^22 rays on the 128^3 torus (config-1 network, random weights biased
    to hit), fused vs two kernels per chunk on the same handle."""
    w = S.WORKLOADS["torus128_query"]
    net = w["net"]
    mesh = S.make_mesh(w["shape"])
    h = nif.Nif(net, mesh, precision=nif.NIF_BF16)
    nif.nif_set_knob(h.h, nif.NIF_KNOB_QUERY_FUSED, 1)
    ws, s = occupancy_biased_weights(net, 312)
    h.set_params(random_tables(net, 311), ws, s)
    rays = torch.from_numpy(S.sphere_rays(1 << 22, seed=313)).to(_dev())
    pose = [(0.6, -0.5, 0.7)]
    a = nif.nif_query(h.h, pose, rays).cpu().numpy().view(nif.HIT_DTYPE).reshape(-1)
    nif.nif_set_knob(h.h, nif.NIF_KNOB_QUERY_FUSED, 0)
    b = nif.nif_query(h.h, pose, rays).cpu().numpy().view(nif.HIT_DTYPE).reshape(-1)
    nif.nif_sync_status(h.h)
    h.close()
    ha, hb = a["hit"] > 0, b["hit"] > 0
    both = ha & hb
    assert ha.sum() > 100_000
    assert both.sum() >= 0.995 * (ha | hb).sum()
    # where both take the same first-hit segment the outputs agree to the
    # 16-bit rounding of an activation; another segment moves D by about a
    # voxel (1/128)
    same = both.copy()
    same[both] = np.abs(a["D"][both] - b["D"][both]) < 2e-3
    assert same.sum() >= 0.99 * both.sum()
    assert np.percentile(np.abs(a["D"][same] - b["D"][same]), 99) < 5e-4
    assert (a["material"][same] == b["material"][same]).mean() > 0.99
    cosang = (a["n"][same] * b["n"][same]).sum(1)
    assert np.percentile(cosang, 1) > np.cos(np.radians(1.0))


def test_fused_query_no_segments_and_small_counts(nif, torus):
    net = S.NetConfig()
    h = nif.Nif(net, torus, precision=nif.NIF_BF16)
    nif.nif_set_knob(h.h, nif.NIF_KNOB_QUERY_FUSED, 1)
    ws, s = occupancy_biased_weights(net, 322)
    h.set_params(random_tables(net, 321), ws, s)
    # rays that start beyond the cube and point away: no segment at all
    far = np.zeros((300, 8), np.float32)
    far[:, 0:3] = 5.0
    far[:, 3:6] = np.array([1.0, 0.0, 0.0], np.float32)
    far[:, 7] = 10.0
    hits = nif.nif_query(h.h, [(0.0, 0.0, 0.0)], torch.from_numpy(far).to(_dev()))
    nif.nif_sync_status(h.h)
    assert int((hits[:, 7].view(torch.int32) & 0xff).ne(0).sum()) == 0
    # 1, 2 and 129 rays: one partial tile, and a tile boundary inside a ray
    tables, ws2, _ = h.get_params()
    pose = (0.2, 0.1, -0.3)
    pool = S.sphere_rays(600, seed=331)
    pool = pool[certain_rays(net.voxel_res, torus, pose, pool)]
    for n in (1, 2, 129):
        rays_np = np.ascontiguousarray(pool[:n])
        hits = nif.nif_query(h.h, [pose], torch.from_numpy(rays_np).to(_dev())).cpu().numpy()
        nif.nif_sync_status(h.h)
        hits = hits.view(nif.HIT_DTYPE).reshape(-1)
        _check_against_oracle(nif, net, torus, hits, tables, [w.astype(np.float64) for w in ws2], pose, rays_np)
    h.close()


@pytest.mark.parametrize("levels,log2T,fused", [(8, 14, True), (16, 16, True), (16, 17, False), (16, 19, False)])
def test_fused_query_applies_to_small_tables(nif, torus, levels, log2T, fused):
    """The fused kernel runs where the FP16 table copy is at most 4 MiB; larger
    tables take the two-kernel path (the profile names the stages that ran)."""
    net = S.NetConfig(levels=levels, log2_table=log2T, mlp_depth=2, mlp_width=32)
    h = nif.Nif(net, torus, precision=nif.NIF_BF16)
    rays = torch.from_numpy(S.sphere_rays(500, seed=341)).to(_dev())
    nif.nif_query(h.h, [(0.1, 0.2, 0.3)], rays)
    nif.nif_profile(h.h, 1)
    nif.nif_query(h.h, [(0.1, 0.2, 0.3)], rays)
    stages = set(nif.nif_profile_read(h.h))
    nif.nif_profile(h.h, 0)
    h.close()
    assert ("encode_mlp_tc" in stages) == fused, stages
    assert ("mlp_fwd_tc" in stages) == (not fused), stages
