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
