"""nif_train_steps (several training steps in one call, each step's batch built
on a second stream while the previous step trains) computes what the same
number of nif_train_step calls computes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2604_24666_gb300 import synth as S

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


@pytest.mark.parametrize("mixed", [False, True])
def test_train_steps_equal_single_steps(nif, torus, mixed):
    net = S.NetConfig()
    kw = dict(precision=nif.NIF_BF16, flags=nif.NIF_FLAG_MIXED_TRAINING) if mixed else {}
    a = nif.Nif(net, torus, seed=7, **kw)
    b = nif.Nif(net, torus, seed=7, **kw)
    n_seg, n_poses = 1 << 14, 8
    # learning rates 0: every step's loss depends only on its batch, so the last
    # batch built beside the previous step must be the one nif_train_step builds
    for K in (1, 2, 5):
        seed = 500 + 10 * K
        la = nif.nif_train_steps(a.h, K, n_seg, n_poses, seed, lr_grid=0.0, lr_mlp=0.0, want_loss=True)
        lb, _ = nif.nif_train_step(b.h, n_seg, n_poses, seed + K - 1, lr_grid=0.0, lr_mlp=0.0, want_loss=True)
        np.testing.assert_allclose(la, lb, rtol=1e-9, atol=1e-12)
    # with learning: the same trajectory up to the order of float atomics
    la = nif.nif_train_steps(a.h, 30, n_seg, n_poses, 900, lr_grid=1e-2, lr_mlp=5e-3, want_loss=True)
    for i in range(30):
        lb, _ = nif.nif_train_step(b.h, n_seg, n_poses, 900 + i, lr_grid=1e-2, lr_mlp=5e-3, want_loss=i == 29)
    np.testing.assert_allclose(la[1:], lb[1:], rtol=5e-2, atol=1e-3)
    a.close()
    b.close()


@pytest.mark.parametrize("mixed", [False, True])
def test_train_steps_rays_equal_single_steps(nif, torus, mixed):
    """nif_train_steps_rays (rays from pinned host memory, copied and batched
    beside the previous step, every step's loss read back) against the same
    steps through nif_train_step_rays; two instances per step."""
    net = S.NetConfig()
    kw = dict(precision=nif.NIF_BF16, flags=nif.NIF_FLAG_MIXED_TRAINING) if mixed else {}
    a = nif.Nif(net, torus, seed=11, **kw)
    b = nif.Nif(net, torus, seed=11, **kw)
    K, per, n_seg = 6, 3000, 1 << 13
    rays = np.stack([np.concatenate([S.sphere_rays(per, seed=700 + 2 * i), S.sphere_rays(per, seed=701 + 2 * i)])
                     for i in range(K)])
    poses = np.stack([S.poses(2, seed=800 + i) for i in range(K)]).astype(np.float32)
    inst = torch.tensor([0, per, 2 * per], dtype=torch.int32, device="cuda")
    rays_host = torch.from_numpy(rays).pin_memory()
    for lr_grid, lr_mlp, rtol in ((0.0, 0.0, 1e-9), (1e-2, 5e-3, 5e-2)):
        la = nif.nif_train_steps_rays(a.h, poses, rays_host, n_seg, inst_offsets=inst, lr_grid=lr_grid,
                                      lr_mlp=lr_mlp)
        lb = np.stack([nif.nif_train_step_rays(b.h, poses[i], torch.from_numpy(rays[i]).cuda(), n_seg,
                                               inst_offsets=inst, lr_grid=lr_grid, lr_mlp=lr_mlp)
                       for i in range(K)])
        assert la.shape == (K, 6) and np.isfinite(la).all()
        # without learning every step's loss is a function of its own batch; with
        # learning the trajectories agree up to the order of float atomics
        np.testing.assert_allclose(la, lb, rtol=rtol, atol=1e-12 if rtol < 1e-6 else 1e-3)
    # no loss requested: enqueued only, then the same state as a synchronised call
    assert nif.nif_train_steps_rays(a.h, poses[:2], rays_host[:2], n_seg, inst_offsets=inst, want_loss=False) is None
    torch.cuda.synchronize()
    a.close()
    b.close()


def test_train_steps_rays_pageable_host_memory(nif, torus):
    """Rays in pageable host memory: the copies serialise with the host but
    the steps compute the same losses as from pinned memory."""
    net = S.NetConfig()
    a = nif.Nif(net, torus, seed=13)
    b = nif.Nif(net, torus, seed=13)
    rays = np.stack([S.sphere_rays(4000, seed=900 + i) for i in range(3)])
    poses = np.stack([S.poses(1, seed=910 + i) for i in range(3)]).astype(np.float32)
    la = nif.nif_train_steps_rays(a.h, poses, torch.from_numpy(rays).pin_memory(), 1 << 13, lr_grid=0.0, lr_mlp=0.0)
    lb = nif.nif_train_steps_rays(b.h, poses, torch.from_numpy(rays), 1 << 13, lr_grid=0.0, lr_mlp=0.0)
    np.testing.assert_allclose(lb, la, rtol=1e-9, atol=1e-12)
    a.close()
    b.close()


def test_train_steps_rays_rejects_bad_arguments(nif, torus):
    a = nif.Nif(S.NetConfig(), torus)
    rays_host = torch.from_numpy(np.stack([S.sphere_rays(100, seed=1)] * 2))
    bad = np.array([[[2.0, 0.0, 0.0]], [[0.0, 0.0, 0.0]]], np.float32)
    with pytest.raises(nif.NifError):
        nif.nif_train_steps_rays(a.h, bad, rays_host, 1000)       # a pose out of range in step 0
    with pytest.raises(nif.NifError):
        nif.nif_train_steps_rays(a.h, np.zeros((2, 2, 3), np.float32), rays_host, 1000)   # n_inst 2, no offsets
    a.close()


@pytest.mark.parametrize("levels,log2T", [(8, 14), (16, 19)])
def test_train_step_table_gradient_matches_stages(nif, torus, levels, log2T):
    """The table gradient of a whole training step equals the stage-by-stage
    one on the same batch. The step's encoding backward takes the list of
    distinct end points, and with 64 MiB tables their rest-space order, from
    the step's forward. One Adam step from zero moments moves every parameter
    by lr * g / (|g| + 1e-15), so the step's table change must be zero exactly
    where the stage gradient is zero and must have its sign where it is
    clearly nonzero."""
    from tests.gpu_common import random_tables
    net = S.NetConfig(levels=levels, log2_table=log2T)
    pose = (0.4, -0.7, 0.3)
    rays_np = S.sphere_rays(3000, seed=321)
    tables = random_tables(net, 322, scale=0.5)
    _, ws, _ = S.init_params(net, seed=323)
    dev = torch.device("cuda:0")
    rays = torch.from_numpy(rays_np).to(dev)
    # stage by stage
    a = nif.Nif(net, torus)
    a.set_params(tables, ws)
    offs, segs = nif.nif_segments(a.h, [pose], rays)
    lin = nif.nif_linearize(a.h, [pose], rays, segs)
    lab = nif.nif_labels(a.h, segs, lin)
    feat = nif.nif_encode_segments(a.h, lin, net.in_dim)
    n = feat.shape[0]
    acts = torch.zeros((net.mlp_depth, n, net.mlp_width), dtype=torch.float32, device=dev)
    out = nif.nif_mlp_forward(a.h, feat, acts=acts)
    nif.nif_zero_grad(a.h)
    _, dout = nif.nif_loss(a.h, out, lab, lin)
    dx = nif.nif_mlp_backward(a.h, feat, acts, dout)
    dtab = torch.zeros((net.levels, 1 << net.log2_table, 2), dtype=torch.float32, device=dev)
    nif.nif_encode_segments_backward(a.h, lin, dx, dtab)
    torch.cuda.synchronize()
    g = dtab.cpu().numpy()
    a.close()
    # one training step on the same rays, every segment in the batch
    b = nif.Nif(net, torus)
    b.set_params(tables, ws)
    t0 = b.get_params()[0].copy()
    lr = 1e-3
    nif.nif_train_step_rays(b.h, [pose], rays, 4 * n + 1024, lr_grid=lr, lr_mlp=0.0)
    delta = t0 - b.get_params()[0]
    b.close()
    assert n > 1000 and np.count_nonzero(g) > 1000
    np.testing.assert_array_equal(delta[g == 0], 0.0)
    big = np.abs(g) > 1e-4 * np.abs(g).max()
    # |delta| is lr up to the FP32 rounding of the parameter update
    np.testing.assert_allclose(np.abs(delta[big]), lr, rtol=1e-3)
    agree = np.sign(delta[big]) == np.sign(g[big])
    assert agree.all(), (np.count_nonzero(~agree), big.sum())


@pytest.mark.parametrize("batch_at,ctas,bwd", [(0, 0, 0), (1, 37, -1), (2, -1, 19), (3, 0, 0), (0, 5, 152)])
def test_train_steps_batch_placement_and_fused_forward(nif, torus, batch_at, ctas, bwd):
    """Where the next batch starts beside a step (NIF_KNOB_BATCH_AT), the
    one-launch FP32 forward (NIF_KNOB_FP32_FUSED), its CTA count beside the
    batch (NIF_KNOB_STEP_FWD_CTAS) and the encoding backward's CTA count
    beside the weight gradients (NIF_KNOB_STEP_BWD_CTAS) change the
    schedule, not the steps: the losses equal those of one launch per layer
    on every SM."""
    net = S.NetConfig(levels=16, log2_table=19, mlp_depth=3, mlp_width=64)
    a = nif.Nif(net, torus, seed=9)
    b = nif.Nif(net, torus, seed=9)
    nif.nif_set_knob(a.h, nif.NIF_KNOB_FP32_FUSED, 0)
    nif.nif_set_knob(a.h, nif.NIF_KNOB_STEP_BWD_CTAS, -1)
    nif.nif_set_knob(b.h, nif.NIF_KNOB_BATCH_AT, batch_at)
    nif.nif_set_knob(b.h, nif.NIF_KNOB_STEP_FWD_CTAS, ctas)
    nif.nif_set_knob(b.h, nif.NIF_KNOB_STEP_BWD_CTAS, bwd)
    # learning rates 0: each step's loss depends only on its batch (a batch
    # built into the buffers of the step still running would show here)
    for K in (1, 3):
        la = nif.nif_train_steps(a.h, K, 1 << 15, 8, 900 + K, lr_grid=0.0, lr_mlp=0.0, want_loss=True)
        lb = nif.nif_train_steps(b.h, K, 1 << 15, 8, 900 + K, lr_grid=0.0, lr_mlp=0.0, want_loss=True)
        np.testing.assert_allclose(lb, la, rtol=1e-6, atol=1e-9)
    # with learning: the same trajectory up to the order of float atomics
    la = nif.nif_train_steps(a.h, 4, 1 << 15, 8, 950, lr_grid=1e-2, lr_mlp=1e-3, want_loss=True)
    lb = nif.nif_train_steps(b.h, 4, 1 << 15, 8, 950, lr_grid=1e-2, lr_mlp=1e-3, want_loss=True)
    np.testing.assert_allclose(lb[1:], la[1:], rtol=1e-2, atol=1e-4)
    a.close()
    b.close()


def test_profile_filter_times_only_named_stages(nif, torus):
    h = nif.Nif(S.NetConfig(), torus, seed=3)
    nif.nif_train_steps(h.h, 1, 1 << 14, 4, 11)
    nif.nif_profile_filter(h.h, ["encode_bwd", "adam"])
    nif.nif_profile(h.h, 1)
    nif.nif_train_steps(h.h, 3, 1 << 14, 4, 12)
    prof = nif.nif_profile_read(h.h)
    nif.nif_profile(h.h, 0)
    assert set(prof) == {"encode_bwd", "adam"}, set(prof)
    assert prof["encode_bwd"][1] == 3 and prof["encode_bwd"][0] > 0
    nif.nif_profile_filter(h.h, None)
    nif.nif_profile(h.h, 1)
    nif.nif_train_steps(h.h, 1, 1 << 14, 4, 13)
    assert len(nif.nif_profile_read(h.h)) > 5
    nif.nif_profile(h.h, 0)
    h.close()


def test_profile_timeline_orders_stages(nif, torus):
    h = nif.Nif(S.NetConfig(), torus, seed=4)
    nif.nif_train_steps(h.h, 1, 1 << 14, 4, 21)
    nif.nif_profile(h.h, 1)
    nif.nif_train_steps(h.h, 2, 1 << 14, 4, 22)
    tl = nif.nif_profile_timeline(h.h)
    prof = nif.nif_profile_read(h.h)
    nif.nif_profile(h.h, 0)
    h.close()
    assert tl[0][1] == 0.0 and all(b >= a for _, a, b in tl)
    names = [n for n, _, _ in tl]
    assert names.count("adam") == 2 and names.count("encode_bwd") == 2
    # the same intervals as the folded sums
    tot = sum(b - a for n, a, b in tl if n == "encode_bwd")
    assert abs(tot - prof["encode_bwd"][0]) < 1e-3 * max(1.0, tot)
    # a step's Adam update follows its encoding backward on the step's stream
    i_bwd = names.index("encode_bwd")
    i_adam = names.index("adam")
    assert tl[i_adam][1] >= tl[i_bwd][2] - 1e-3


@pytest.mark.parametrize("batch_at", [0, 1])
def test_deferred_weight_update_trains_alike(nif, torus, batch_at):
    """FP32 steps whose weights are updated on the second stream beside the
    next step (NIF_KNOB_DEFER_WEIGHTS) follow the trajectory of steps that
    update everything at once, and the parameters after the call are final:
    losses of 12 pipelined steps agree up to the order of float atomics, and
    the weights read back right after the call equal those of a handle that
    trained the same steps one call at a time."""
    net = S.NetConfig(levels=16, log2_table=16, mlp_depth=3, mlp_width=64)
    a = nif.Nif(net, torus, seed=19)
    b = nif.Nif(net, torus, seed=19)
    for h, d in ((a, 1), (b, 0)):
        nif.nif_set_knob(h.h, nif.NIF_KNOB_DEFER_WEIGHTS, d)
        nif.nif_set_knob(h.h, nif.NIF_KNOB_BATCH_AT, batch_at)
    # learning rates 0: the batches alone decide the losses
    la = nif.nif_train_steps(a.h, 3, 1 << 15, 8, 700, lr_grid=0.0, lr_mlp=0.0, want_loss=True)
    lb = nif.nif_train_steps(b.h, 3, 1 << 15, 8, 700, lr_grid=0.0, lr_mlp=0.0, want_loss=True)
    np.testing.assert_allclose(la, lb, rtol=1e-6, atol=1e-9)
    la = nif.nif_train_steps(a.h, 12, 1 << 15, 8, 800, lr_grid=1e-2, lr_mlp=1e-3, want_loss=True)
    lb = nif.nif_train_steps(b.h, 12, 1 << 15, 8, 800, lr_grid=1e-2, lr_mlp=1e-3, want_loss=True)
    np.testing.assert_allclose(la[1:], lb[1:], rtol=2e-2, atol=1e-4)
    # a single step with lr 0 then reads the updated weights: a stale copy
    # (the last update still running) would change this loss
    ta, wa, _ = a.get_params()
    tb, wb, _ = b.get_params()
    for x, y in zip(wa, wb):
        np.testing.assert_allclose(x, y, rtol=5e-2, atol=1e-3)
    l1 = nif.nif_train_steps(a.h, 1, 1 << 15, 8, 900, lr_grid=0.0, lr_mlp=0.0, want_loss=True)
    l2, _ = nif.nif_train_step(a.h, 1 << 15, 8, 900, lr_grid=0.0, lr_mlp=0.0, want_loss=True)
    np.testing.assert_allclose(l1, l2, rtol=1e-6, atol=1e-9)
    a.close()
    b.close()


def test_high_priority_streams_compute_the_same(nif, torus):
    """NIF_KNOB_STEP_PRIORITY moves the steps onto the handle's high-priority
    streams (joined back into the caller's): the same batches and losses."""
    net = S.NetConfig()
    a = nif.Nif(net, torus, seed=23)
    b = nif.Nif(net, torus, seed=23)
    nif.nif_set_knob(b.h, nif.NIF_KNOB_STEP_PRIORITY, 1)
    for K in (1, 4):
        la = nif.nif_train_steps(a.h, K, 1 << 14, 8, 600 + K, lr_grid=0.0, lr_mlp=0.0, want_loss=True)
        lb = nif.nif_train_steps(b.h, K, 1 << 14, 8, 600 + K, lr_grid=0.0, lr_mlp=0.0, want_loss=True)
        np.testing.assert_allclose(la, lb, rtol=1e-6, atol=1e-9)
    # the caller's stream is ordered after the call: parameters read back at once
    la = nif.nif_train_steps(a.h, 6, 1 << 14, 8, 650, lr_grid=1e-2, lr_mlp=5e-3, want_loss=True)
    lb = nif.nif_train_steps(b.h, 6, 1 << 14, 8, 650, lr_grid=1e-2, lr_mlp=5e-3, want_loss=True)
    np.testing.assert_allclose(la[1:], lb[1:], rtol=2e-2, atol=1e-4)
    _, wa, _ = a.get_params()
    _, wb, _ = b.get_params()
    for x, y in zip(wa, wb):
        np.testing.assert_allclose(x, y, rtol=5e-2, atol=1e-3)
    a.close()
    b.close()
