"""Pieces of the animated frame loop on the GPU: shadow rays from primary
hits, the pose-fitting gradient step against the oracle, and query plans
that stay valid while other calls grow the handle's scratch buffers."""
import numpy as np
import pytest
import torch

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


def _hit_fields(nif, hits):
    return hits.cpu().numpy().view(nif.HIT_DTYPE).reshape(-1)


def test_shadow_rays_from_hits(nif, torus):
    net = S.NetConfig()
    h = nif.Nif(net, torus)
    h.set_params(random_tables(net, 181), *occupancy_biased_weights(net, 182))
    rays_np = S.sphere_rays(3000, seed=183)
    rays = torch.from_numpy(rays_np).cuda()
    pose = (0.3, -0.5, 0.2)
    hits = nif.nif_query(h.h, [pose], rays)
    light = np.array([0.4, 0.3, 0.87])
    sh = nif.nif_shadow_rays(h.h, rays, hits, light, eps=1e-3, tmax=3.0).cpu().numpy()
    hf = _hit_fields(nif, hits)
    hit = hf["hit"] > 0
    assert 0 < hit.sum() < len(hit)
    L = (light / np.linalg.norm(light)).astype(np.float32)
    np.testing.assert_allclose(sh[:, 3:6], np.broadcast_to(L, (len(sh), 3)), rtol=1e-6, atol=1e-7)
    o = rays_np[:, 0:3] + hf["D"][:, None] * rays_np[:, 3:6]
    np.testing.assert_allclose(sh[hit, 0:3], o[hit], atol=2e-6)
    assert np.all(sh[hit, 6] == np.float32(1e-3)) and np.all(sh[hit, 7] == np.float32(3.0))
    assert np.all(sh[~hit, 6] == 0) and np.all(sh[~hit, 7] == 0)
    # occlusion queries on them: misses stay misses
    occl = _hit_fields(nif, nif.nif_query(h.h, [pose], torch.from_numpy(sh).cuda(), flags=nif.NIF_SHADOW_ONLY))
    assert not np.any(occl["hit"][~hit])
    h.close()


def _pose_step_oracle(net, mesh, tables, ws, s, poses, parts):
    """dL/dposes of the task loss by the oracle on the segments of each ray set."""
    N = net.voxel_res
    occ, ptr, idx = O.voxelize(N, mesh)
    segs, p0s, p1s, lrs, labs = [], [], [], [], []
    for pose, r in zip(poses, parts):
        seg = O.segments(N, occ, pose, r)
        p0, p1, _, lr = O.linearize(pose, r, seg)
        segs.append(seg); p0s.append(p0); p1s.append(p1); lrs.append(lr)
        labs.append(O.labels(mesh, ptr, idx, seg.vox, p0, p1))
    p0 = np.concatenate(p0s); p1 = np.concatenate(p1s); lr = np.concatenate(lrs)
    lab = {k: np.concatenate([l[k] for l in labs]) for k in labs[0]}
    x = O.encode_segments(net, tables, p0, p1)
    out, acts = O.mlp_forward(ws, x)
    tot, parts_, dout, _ = O.loss(net, out, lab, s, lr)
    _, dx = O.mlp_backward(ws, acts, dout)
    ref = np.zeros((len(poses), 3))
    start = 0
    for i, pose in enumerate(poses):
        m = len(segs[i])
        ref[i] = O.pose_gradient(net, tables, pose, p0s[i], p1s[i], dx[start:start + m])
        start += m
    return ref, tot


def test_pose_step_matches_oracle(nif, torus):
    net = S.NetConfig(levels=8, log2_table=12)
    N = net.voxel_res
    poses = np.array([[0.5, -0.9, 0.4], [-0.7, 0.6, -0.3]], np.float32)
    parts = []
    for i, seed in enumerate((191, 192)):
        r = S.sphere_rays(900, seed=seed)
        parts.append(r[certain_rays(N, torus, poses[i], r, with_labels=True)])
    rays_np = np.concatenate(parts)
    inst = np.array([0, len(parts[0]), len(rays_np)], np.int32)
    h = nif.Nif(net, torus)
    tables = random_tables(net, 193, scale=0.5)
    _, ws, _ = S.init_params(net, seed=194)
    s = np.array([0.1, -0.2, 0.0, 0.3, -0.1], np.float32)
    h.set_params(tables, ws, s)
    rays = torch.from_numpy(rays_np).cuda()
    it = torch.from_numpy(inst).cuda()
    nif.nif_zero_grad(h.h)
    dposes, parts_gpu = nif.nif_pose_step(h.h, poses, rays, 1 << 20, inst_offsets=it, want_loss=True)
    ref, tot = _pose_step_oracle(net, torus, tables, ws, s, poses, parts)
    np.testing.assert_allclose(dposes.cpu().numpy(), ref, rtol=5e-3, atol=5e-3 * np.abs(ref).max())
    assert abs(parts_gpu[0] - tot) < 1e-4 * max(1.0, abs(tot))
    gt, gw, gs = h.get_grads()                # nothing added to the training gradient
    assert not gt.any() and not any(w.any() for w in gw) and not gs.any()
    h.close()


def _rnd(dt):
    return lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(dt).to(torch.float64).numpy()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_pose_step_mixed_precision_matches_rounded_oracle(nif, torus, prec):
    """16-bit pose step against the oracle with the path's storage points
    rounded: FP16 table copy, 16-bit features, weights, activations and
    loss-scaled output gradients (S = 2^15 for FP16, 1 for BF16); the
    encoding's dL/dp uses the FP32 tables on both sides. What remains is FP32
    against FP64 accumulation and the rare one-ulp 16-bit rounding flip it
    causes; a flip that moves a predicted distance across the ReLU head's
    zero, or a segment with d near 0 where the log-distance gradient is
    ~1/(d + eps), shifts one segment's whole term. Bound: 2 % (FP16) / 6 %
    (BF16, 8 significant bits; measured 3 %) of the largest component."""
    net = S.NetConfig(levels=8, log2_table=12)
    N = net.voxel_res
    dt = torch.bfloat16 if prec == "bf16" else torch.float16
    p = nif.NIF_BF16 if prec == "bf16" else nif.NIF_FP16
    poses = np.array([[0.5, -0.9, 0.4], [-0.7, 0.6, -0.3]], np.float32)
    parts = []
    for i, seed in enumerate((211, 212)):
        r = S.sphere_rays(900, seed=seed)
        parts.append(r[certain_rays(N, torus, poses[i], r, with_labels=True)])
    rays_np = np.concatenate(parts)
    inst = np.array([0, len(parts[0]), len(rays_np)], np.int32)
    h = nif.Nif(net, torus, precision=p)
    tables = random_tables(net, 213, scale=0.5)
    _, ws, _ = S.init_params(net, seed=214)
    s = np.array([0.1, -0.2, 0.0, 0.3, -0.1], np.float32)
    h.set_params(tables, ws, s)
    scale, _ = nif.nif_loss_scale(h.h)
    dposes, _ = nif.nif_pose_step(h.h, poses, torch.from_numpy(rays_np).cuda(), 1 << 20,
                                  inst_offsets=torch.from_numpy(inst).cuda())
    rnd = _rnd(dt)
    occ, ptr, idx = O.voxelize(N, torus)
    segs, p0s, p1s, lrs, labs = [], [], [], [], []
    for pose, r in zip(poses, parts):
        seg = O.segments(N, occ, pose, r)
        p0, p1, _, lr = O.linearize(pose, r, seg)
        segs.append(len(seg)); p0s.append(p0); p1s.append(p1); lrs.append(lr)
        labs.append(O.labels(torus, ptr, idx, seg.vox, p0, p1))
    lab = {k: np.concatenate([l[k] for l in labs]) for k in labs[0]}
    t16 = _rnd(torch.float16)(tables)
    x = rnd(O.encode_segments(net, t16, np.concatenate(p0s), np.concatenate(p1s)))
    out, acts = O.mlp_forward_rounded(ws, x, rnd)
    _, _, dout, _ = O.loss(net, out, lab, s, np.concatenate(lrs))
    _, dx = O.mlp_backward_rounded(ws, acts, dout, scale, rnd)
    dx = dx / scale
    ref = np.zeros((2, 3))
    start = 0
    for i in range(2):
        ref[i] = O.pose_gradient(net, tables, poses[i], p0s[i], p1s[i], dx[start:start + segs[i]])
        start += segs[i]
    got = dposes.cpu().numpy()
    tol = 2e-2 if prec == "fp16" else 6e-2
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (got, ref)
    h.close()


def test_query_plan_survives_scratch_growth(nif, torus):
    net = S.NetConfig()
    h = nif.Nif(net, torus, precision=nif.NIF_BF16)
    h.set_params(random_tables(net, 201), *occupancy_biased_weights(net, 202))
    rays = torch.from_numpy(S.sphere_rays(2000, seed=203)).cuda()
    hits = torch.zeros((2000, 8), dtype=torch.float32, device="cuda")
    pose = [(0.2, 0.7, -0.4)]
    plan = nif.QueryPlan(h.h, pose, rays, hits, autotune=False)
    plan.run(pose)
    ref = nif.nif_query(h.h, pose, rays)
    torch.cuda.synchronize()
    assert torch.equal(hits.view(torch.int32), ref.view(torch.int32))
    # calls that grow every scratch buffer and the instance buffers
    big = torch.from_numpy(S.sphere_rays(200000, seed=204)).cuda()
    nif.nif_query(h.h, S.poses(8, seed=205), big,
                  inst_offsets=torch.arange(0, 200001, 25000, dtype=torch.int32).cuda())
    nif.nif_train_step(h.h, 1 << 16, 4, 7, want_loss=False)       # new weights as well
    hits.zero_()
    plan.run(pose)
    nif.nif_sync_status(h.h)
    ref = nif.nif_query(h.h, pose, rays)
    torch.cuda.synchronize()
    assert torch.equal(hits.view(torch.int32), ref.view(torch.int32))
    plan.close()
    h.close()
