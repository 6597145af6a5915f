"""nif_query keeps its counts on the device and does not block the host.

* With a long kernel ahead of it on the stream, the call returns before that
  kernel ends, and its result equals a query run alone.
* A query whose segments exceed its capacity (sized from an initial
  estimate the test sets far too low) answers the rays whose segment lists
  fit, reports no hit for the others and latches NIF_ERR_CAPACITY; the next
  query, sized from the total the first one sent back, answers every ray.
"""
import time

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


def _handle(nif, prec):
    net = S.NetConfig()
    h = nif.Nif(net, S.torus_mesh(), precision=prec)
    ws, s = occupancy_biased_weights(net, 502)
    h.set_params(random_tables(net, 501), ws, s)
    return h


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_query_returns_before_the_stream_is_done(nif, prec):
    p = nif.NIF_FP32 if prec == "fp32" else nif.NIF_BF16
    h = _handle(nif, p)
    dev = torch.device("cuda:0")
    rays = torch.from_numpy(S.sphere_rays(1 << 16, seed=503)).to(dev)
    pose = [(0.3, -0.6, 0.2)]
    ref = nif.nif_query(h.h, pose, rays)           # sizes every buffer
    nif.nif_sync_status(h.h)
    hits = torch.zeros_like(ref)
    torch.cuda._sleep(500_000_000)                 # ~0.25 s of GPU time ahead of the query
    t0 = time.perf_counter()
    nif.nif_query(h.h, pose, rays, hits=hits)
    dt = time.perf_counter() - t0
    torch.cuda.synchronize()
    assert dt < 0.05, dt
    assert torch.equal(hits.view(torch.int32), ref.view(torch.int32))
    h.close()


def test_query_capacity_overflow_then_recovers(nif):
    dev = torch.device("cuda:0")
    rays = torch.from_numpy(S.sphere_rays(100_000, seed=511)).to(dev)
    pose = [(0.5, 0.4, -0.3)]
    a = _handle(nif, nif.NIF_FP32)
    ref = nif.nif_query(a.h, pose, rays)
    nif.nif_sync_status(a.h)
    a.close()
    h = _handle(nif, nif.NIF_FP32)
    nif.nif_set_knob(h.h, nif.NIF_KNOB_QUERY_SEGS, 0.1)       # capacity 10,000 segments
    hits = nif.nif_query(h.h, pose, rays)
    with pytest.raises(nif.NifError) as e:
        nif.nif_sync_status(h.h)
    assert e.value.status == nif.NIF_ERR_CAPACITY
    got = hits.view(torch.int32).cpu().numpy()
    want = ref.view(torch.int32).cpu().numpy()
    same = np.all(got == want, axis=1)
    k = int(np.argmin(same)) if not same.all() else len(same)
    assert 0 < k < len(same)                        # a prefix of whole rays was answered exactly
    assert np.all((got[k:, 7] & 0xff) == 0)         # the rest report no hit
    hits2 = nif.nif_query(h.h, pose, rays)          # sized from the first query's total
    nif.nif_sync_status(h.h)
    assert torch.equal(hits2.view(torch.int32), ref.view(torch.int32))
    h.close()
