"""Failure paths of the library, made on the host: no kernel is broken, no
address is bad, and every wait that a test makes run out is bounded.

* A bounded mbarrier wait of a tensor-core kernel runs out when the handle's
  wait bound is set far below what the pipeline needs: the launch latches
  NIF_ERR_TIMEOUT, drains its own copies and MMAs, frees its tensor memory,
  and the handle gives correct results again once the bound is restored.
* The single-traversal segment scratch overflows when the test shrinks it:
  the device-gated second traversal must give the same segments, query
  results and training losses as the normal path.
* A segment capacity that is too small returns (or, in a query plan,
  latches) NIF_ERR_CAPACITY and writes nothing past it.
* A non-finite parameter makes a training step report NIF_ERR_NAN.
* An allocation made to fail on the host (NIF_KNOB_FAIL_ALLOC) returns
  NIF_ERR_OOM; the handle recovers with the results, and the training state,
  of a handle that never failed.
* A loss scale far too large makes FP16 steps overflow one after another:
  each is skipped and halves the scale until steps are taken again.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2604_24666_gb300 import synth as S
from tests.gpu_common import occupancy_biased_weights, random_tables

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


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_wait_bound_expires_then_handle_recovers(nif, torus, prec):
    net = S.NetConfig(levels=16, log2_table=14, mlp_depth=3, mlp_width=64)
    p = nif.NIF_BF16 if prec == "bf16" else nif.NIF_FP32
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    h = nif.Nif(net, torus, precision=p)
    tables, ws, s = S.init_params(net, seed=301)
    h.set_params(tables, ws, s)
    n = 1 << 20
    g = torch.Generator(device=_dev()).manual_seed(302)
    x = torch.randn((n, net.in_dim), generator=g, device=_dev()).to(dt)
    ref = nif.nif_mlp_forward(h.h, x, precision=p)
    nif.nif_sync_status(h.h)
    # 1 ns: a wait that does not complete within the hardware's own try-wait
    # window gives up at once
    nif.nif_set_knob(h.h, nif.NIF_KNOB_WAIT_NS, 1)
    nif.nif_mlp_forward(h.h, x, precision=p)
    with pytest.raises(nif.NifError) as e:
        nif.nif_sync_status(h.h)
    assert e.value.status == nif.NIF_ERR_TIMEOUT
    nif.nif_sync_status(h.h)                       # the status word was read and cleared
    nif.nif_set_knob(h.h, nif.NIF_KNOB_WAIT_NS, 0)
    got = nif.nif_mlp_forward(h.h, x, precision=p)
    nif.nif_sync_status(h.h)
    assert torch.equal(got, ref)
    with pytest.raises(nif.NifError) as e:
        nif.nif_set_knob(h.h, nif.NIF_KNOB_WAIT_NS, -1)
    assert e.value.status == nif.NIF_ERR_ARG
    h.close()


def test_query_through_segment_scratch_overflow(nif, torus):
    net = S.NetConfig()
    tables = random_tables(net, 311)
    ws, s = occupancy_biased_weights(net, 312)
    rays = torch.from_numpy(S.sphere_rays(6000, seed=313)).to(_dev())
    pose = [(0.5, -0.7, 0.3)]
    out = []
    for scale in (1.0, 1e-3):
        h = nif.Nif(net, torus)
        h.set_params(tables, ws, s)
        nif.nif_set_knob(h.h, nif.NIF_KNOB_SEG_SCRATCH, scale)
        offs, segs = nif.nif_segments(h.h, pose, rays)
        hits = nif.nif_query(h.h, pose, rays)
        nif.nif_sync_status(h.h)
        out.append((offs, segs, hits))
        h.close()
    assert out[0][1].shape[0] > 4096 + 1000          # more segments than the shrunk scratch holds
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert torch.equal(out[0][2].view(torch.int32), out[1][2].view(torch.int32))
    assert int((out[0][2][:, 7].view(torch.int32) & 0xff).ne(0).sum()) > 100


def test_training_batch_through_segment_scratch_overflow(nif, torus):
    net = S.NetConfig()
    tables, ws, s = S.init_params(net, seed=321)
    rays = torch.from_numpy(S.sphere_rays(8000, seed=322)).to(_dev())
    poses = S.poses(4, seed=323)
    inst = torch.tensor([0, 2000, 4000, 6000, 8000], dtype=torch.int32, device=_dev())
    losses = []
    for scale in (1.0, 1e-3):
        h = nif.Nif(net, torus)
        h.set_params(tables, ws, s)
        nif.nif_set_knob(h.h, nif.NIF_KNOB_SEG_SCRATCH, scale)
        loss = nif.nif_train_step_rays(h.h, poses, rays, 1 << 14, inst_offsets=inst)
        losses.append(np.asarray(loss))
        h.close()
    # the same batch: the loss parts agree to the order of their FP64 accumulation
    np.testing.assert_allclose(losses[0], losses[1], rtol=1e-9, atol=1e-12)


def test_segment_capacity_errors(nif, torus):
    net = S.NetConfig()
    h = nif.Nif(net, torus)
    rays = torch.from_numpy(S.sphere_rays(2000, seed=331)).to(_dev())
    pose = [(0.2, 0.4, -0.3)]
    offs, segs = nif.nif_segments(h.h, pose, rays)
    total = segs.shape[0]
    cap = total // 2
    buf = torch.full((cap + 64, 4), -1, dtype=torch.int32, device=_dev())
    o2 = torch.zeros_like(offs)
    p, n_inst = nif._poses(pose)
    got = nif._i64()
    st = nif.lib().nif_segments(h.h, p, n_inst, nif._ptr(rays), None, rays.shape[0], nif._ptr(o2), nif._ptr(buf),
                                cap, ctypes.byref(got), nif._stream(None))
    torch.cuda.synchronize()
    assert st == nif.NIF_ERR_CAPACITY and got.value == total
    assert torch.equal(o2, offs)
    assert bool((buf[cap:] == -1).all())            # nothing written past the capacity
    # a query plan whose capacity is too small latches the error on the device
    hits = torch.zeros((rays.shape[0], 8), dtype=torch.float32, device=_dev())
    plan = nif.QueryPlan(h.h, pose, rays, hits, seg_capacity=cap, autotune=False)
    plan.run(pose)
    with pytest.raises(nif.NifError) as e:
        nif.nif_sync_status(h.h)
    assert e.value.status == nif.NIF_ERR_CAPACITY
    plan.close()
    h.close()


def test_non_finite_parameter_reports_nan(nif, torus):
    net = S.NetConfig()
    h = nif.Nif(net, torus, seed=5)
    tables, ws, s = h.get_params()
    bad = [w.copy() for w in ws]
    bad[-1][0, 3] = np.nan                          # occupancy logit weight
    h.set_params(tables, bad, s)
    with pytest.raises(nif.NifError) as e:
        nif.nif_train_step(h.h, 1 << 13, 4, 341)
    assert e.value.status == nif.NIF_ERR_NAN
    # restored parameters train again
    h.set_params(tables, ws, s)
    nif.nif_reset_optimizer(h.h)
    loss, _ = nif.nif_train_step(h.h, 1 << 13, 4, 342)
    assert np.all(np.isfinite(loss))
    h.close()


def test_injected_allocation_failure_query_recovers(nif, torus):
    """Each of a fresh handle's first scratch allocations fails in turn
    (NIF_KNOB_FAIL_ALLOC, an out-of-memory cudaMalloc made on the host): the
    query returns NIF_ERR_OOM, and the same query on the same handle then
    gives bit for bit the hits of a handle that never failed."""
    net = S.NetConfig()
    tables, ws, s = S.init_params(net, seed=351)
    rays = torch.from_numpy(S.sphere_rays(4096, seed=352)).to(_dev())
    pose = [(0.3, -0.5, 0.2)]
    ref_h = nif.Nif(net, torus)
    ref_h.set_params(tables, ws, s)
    ref = nif.nif_query(ref_h.h, pose, rays).clone()
    torch.cuda.synchronize()
    failed = []
    for k in range(1, 9):
        h = nif.Nif(net, torus)
        h.set_params(tables, ws, s)
        nif.nif_set_knob(h.h, nif.NIF_KNOB_FAIL_ALLOC, k)
        try:
            nif.nif_query(h.h, pose, rays)
            torch.cuda.synchronize()
        except nif.NifError as e:
            assert e.status == nif.NIF_ERR_OOM, e
            failed.append(k)
        nif.nif_set_knob(h.h, nif.NIF_KNOB_FAIL_ALLOC, 0)
        got = nif.nif_query(h.h, pose, rays)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), k
        h.close()
    assert failed and failed[0] == 1, failed
    ref_h.close()


def _grads_zero(h):
    t, w, s = h.get_grads()
    return not np.any(t) and all(not np.any(x) for x in w) and not np.any(s)


@pytest.mark.parametrize("mixed", [False, True], ids=["fp32", "bf16-mixed"])
def test_injected_allocation_failure_training_recovers(nif, torus, mixed):
    """A training step whose k-th scratch allocation fails returns
    NIF_ERR_OOM and leaves parameters, Adam state and gradients as they were
    (gradients it had added are cleared). With deterministic gradients the
    steps that follow are then bit for bit those of a handle that never
    failed."""
    net = S.NetConfig(levels=8, log2_table=12)
    kw = dict(precision=nif.NIF_BF16, flags=nif.NIF_FLAG_MIXED_TRAINING) if mixed else {}

    def fresh():
        x = nif.Nif(net, torus, seed=3, **kw)
        nif.nif_set_knob(x.h, nif.NIF_KNOB_DETERMINISTIC, 1)
        return x

    ref = fresh()
    for i in range(2):
        nif.nif_train_step(ref.h, 1 << 13, 4, 400 + i)
    want = nif.nif_checkpoint_save(ref.h)
    ref.close()
    failed = []
    for k in (1, 2, 3, 4, 6, 8, 11, 14, 18, 23):
        h = fresh()
        blob0 = nif.nif_checkpoint_save(h.h)
        nif.nif_set_knob(h.h, nif.NIF_KNOB_FAIL_ALLOC, k)
        try:
            nif.nif_train_step(h.h, 1 << 13, 4, 400)
            redo = False
        except nif.NifError as e:
            assert e.status == nif.NIF_ERR_OOM, e
            failed.append(k)
            assert nif.nif_checkpoint_save(h.h) == blob0
            assert _grads_zero(h)
            redo = True
        nif.nif_set_knob(h.h, nif.NIF_KNOB_FAIL_ALLOC, 0)
        if redo:
            nif.nif_train_step(h.h, 1 << 13, 4, 400)
        nif.nif_train_step(h.h, 1 << 13, 4, 401)
        assert nif.nif_checkpoint_save(h.h) == want, k
        h.close()
    assert len(failed) >= 3, failed


def test_loss_scale_overflow_storm(nif, torus):
    """FP16 steps with a loss scale far too large overflow one after another:
    each is skipped (parameters unchanged, the skip counted) and halves the
    scale, until the scale fits and steps are taken again with finite
    parameters."""
    net = S.NetConfig()
    h = nif.Nif(net, torus, precision=nif.NIF_FP16, seed=7, flags=nif.NIF_FLAG_MIXED_TRAINING)
    nif.nif_set_loss_scale(h.h, 2.0 ** 40)
    scale, skipped = nif.nif_loss_scale(h.h)
    assert scale == 2.0 ** 40 and skipped == 0
    taken = None
    for i in range(60):
        before = h.get_params()
        nif.nif_train_step(h.h, 1 << 13, 4, 500 + i, want_loss=False)
        sc, sk = nif.nif_loss_scale(h.h)
        after = h.get_params()
        if sk == skipped + 1:
            assert sc == scale / 2
            assert np.array_equal(after[0], before[0]) and all(np.array_equal(a, b) for a, b in zip(after[1], before[1]))
        else:
            assert sk == skipped and sc == scale
            assert not np.array_equal(after[0], before[0])
            taken = i
            break
        scale, skipped = sc, sk
    assert taken is not None and taken >= 3, (taken, scale)
    t, w, s = h.get_params()
    assert np.isfinite(t).all() and all(np.isfinite(x).all() for x in w) and np.isfinite(s).all()
    h.close()
