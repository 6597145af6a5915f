"""Deterministic gradients (NIF_KNOB_DETERMINISTIC) and bit-identical resume.

By default the library adds gradients with float reductions in L2, whose
order varies from run to run, so two runs of the same steps agree only to
rounding. With the knob set, the table gradient is summed as 64-bit fixed
point (integer addition does not depend on the order), the weight gradients
per row range with the ranges added in order, and the loss sums in block
order. Then:

* the same steps on two handles of the same seed give byte-identical
  checkpoints (parameters, Adam moments, step count, loss-scale state) and
  identical losses, on the FP32 and on the mixed-precision path;
* a checkpoint loaded into a fresh handle continues bit for bit as the
  uninterrupted run does;
* nif_train_steps (next batch built beside each step, weights updated on the
  second stream) equals the same number of nif_train_step calls bit for bit,
  at the training workload's sizes.

How close the deterministic gradients are to the oracle's is checked element
by element in tests/test_gpu_parity.py and tests/test_gpu_parity_full.py.
"""
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


def _kw(nif, mixed):
    return dict(precision=nif.NIF_BF16, flags=nif.NIF_FLAG_MIXED_TRAINING) if mixed else {}


def _det_handle(nif, net, mesh, seed, mixed):
    h = nif.Nif(net, mesh, seed=seed, **_kw(nif, mixed))
    nif.nif_set_knob(h.h, nif.NIF_KNOB_DETERMINISTIC, 1)
    return h


def _steps(nif, h, seeds, n_seg=1 << 13, n_poses=4):
    return np.stack([nif.nif_train_step(h.h, n_seg, n_poses, sd, want_loss=True)[0] for sd in seeds])


@pytest.mark.parametrize("mixed", [False, True], ids=["fp32", "bf16-mixed"])
def test_deterministic_steps_repeat_bit_for_bit(nif, torus, mixed):
    net = S.NetConfig(levels=8, log2_table=12)
    a = _det_handle(nif, net, torus, 3, mixed)
    b = _det_handle(nif, net, torus, 3, mixed)
    la = _steps(nif, a, range(100, 104))
    lb = _steps(nif, b, range(100, 104))
    assert np.array_equal(la, lb)
    assert nif.nif_checkpoint_save(a.h) == nif.nif_checkpoint_save(b.h)
    a.close()
    b.close()


@pytest.mark.parametrize("mixed", [False, True], ids=["fp32", "bf16-mixed"])
def test_checkpoint_resume_is_bit_identical(nif, torus, mixed):
    net = S.NetConfig(levels=8, log2_table=12)
    a = _det_handle(nif, net, torus, 3, mixed)
    _steps(nif, a, range(200, 205))
    blob = nif.nif_checkpoint_save(a.h)
    la = _steps(nif, a, range(205, 208))
    # a fresh handle of another seed, resumed from the checkpoint
    b = _det_handle(nif, net, torus, 99, mixed)
    nif.nif_checkpoint_load(b.h, blob)
    assert nif.nif_checkpoint_save(b.h) == blob
    lb = _steps(nif, b, range(205, 208))
    assert np.array_equal(la, lb)
    assert nif.nif_checkpoint_save(a.h) == nif.nif_checkpoint_save(b.h)
    if mixed:
        assert nif.nif_loss_scale(a.h) == nif.nif_loss_scale(b.h)
    a.close()
    b.close()


@pytest.mark.parametrize("split", [1, 2], ids=["levels-together", "level-halves"])
def test_pipelined_steps_equal_single_steps_bit_for_bit(nif, split):
    """Three steps of the training workload (64^3 ellipsoid union, L = 16,
    T = 2^19, 2^18 segments, 16 poses) through one nif_train_steps call and
    through three nif_train_step calls (the encoding backward's walk with
    its levels together or in halves, NIF_KNOB_BWD_SPLIT)."""
    wl = S.WORKLOADS["ellipsoids64_train"]
    net = wl["net"]
    mesh = S.ellipsoid_union_mesh()
    a = _det_handle(nif, net, mesh, 5, False)
    b = _det_handle(nif, net, mesh, 5, False)
    for x in (a, b):
        nif.nif_set_knob(x.h, nif.NIF_KNOB_BWD_SPLIT, split)
    n_seg, n_poses, seed = 1 << 18, 16, 900
    la = nif.nif_train_steps(a.h, 3, n_seg, n_poses, seed, lr_grid=1e-2, lr_mlp=1e-3, want_loss=True)
    lb = None
    for i in range(3):
        lb, _ = nif.nif_train_step(b.h, n_seg, n_poses, seed + i, lr_grid=1e-2, lr_mlp=1e-3, want_loss=True)
    assert np.array_equal(la, lb)
    assert nif.nif_checkpoint_save(a.h) == nif.nif_checkpoint_save(b.h)
    a.close()
    b.close()


def test_default_mode_differs_only_by_rounding(nif, torus):
    """The knob changes the order of the sums, not what is summed: one step
    from the same state with and without it gives the same loss to FP32
    rounding and nearly the same parameters (an entry whose tiny gradient
    changes sign on its first Adam step moves by 2 lr, which only a handful
    may do)."""
    net = S.NetConfig(levels=8, log2_table=12)
    a = nif.Nif(net, torus, seed=3)
    b = _det_handle(nif, net, torus, 3, False)
    la = _steps(nif, a, [300])
    lb = _steps(nif, b, [300])
    np.testing.assert_allclose(la, lb, rtol=1e-6)
    ta, wa, _ = a.get_params()
    tb, wb, _ = b.get_params()
    assert np.mean(np.abs(tb - ta) > 1e-6) < 1e-3
    for x, y in zip(wa, wb):
        np.testing.assert_allclose(y, x, atol=1e-5)
    with pytest.raises(nif.NifError):
        nif.nif_set_knob(a.h, nif.NIF_KNOB_DETERMINISTIC, 2)
    cat = nif.Nif(S.NetConfig(levels=8, log2_table=12, encoding="concat"), torus)
    with pytest.raises(nif.NifError) as e:
        nif.nif_set_knob(cat.h, nif.NIF_KNOB_DETERMINISTIC, 1)
    assert e.value.status == nif.NIF_ERR_ARG
    for x in (a, b, cat):
        x.close()
