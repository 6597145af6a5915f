"""The allocation-free segment entry point agrees with nif_segments.

nif_segments_noalloc serves callers that cannot allocate device memory (an
application that owns every device allocation through its own allocator, or
a latency-critical loop that must not trigger cudaMalloc's device-wide
synchronisation). Its scratch is a static device array, so this test calls it
twice in a row, on different rays and poses, through the C ABI, and compares
each result with the allocating nif_segments, which runs the same kernels:
offsets and segments must be identical. This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nif():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_24666_gb300 import build
    build.build()
    from paper_2604_24666_gb300 import nif as N
    N.lib()
    return N


def test_segments_noalloc_matches_allocating_entry_point(nif):
    from paper_2604_24666_gb300 import synth as S
    dev = torch.device("cuda:0")
    h = nif.Nif(S.NetConfig(voxel_res=16), S.torus_mesh())
    for call, (pose, seed, n) in enumerate([((0.4, -0.7, 0.3), 1, 3000), ((-0.9, 1.2, 0.8), 2, 1777)]):
        rays = torch.from_numpy(S.sphere_rays(n, seed=seed)).to(dev)
        ref_off, ref_segs = nif.nif_segments(h.h, [pose], rays)
        off = torch.full((n + 1,), -1, dtype=torch.int32, device=dev)
        segs = torch.full((ref_segs.shape[0] + 16, 4), -1, dtype=torch.int32, device=dev)
        total = nif.nif_segments_noalloc(h.h, [pose], rays, off, segs)
        torch.cuda.synchronize()
        assert total == ref_segs.shape[0] > 0, call
        assert torch.equal(off, ref_off), call
        assert torch.equal(segs[:total], ref_segs), call
    # sizes beyond the static scratch are rejected with a clear error
    big = torch.zeros(((1 << 20) + 1, 8), dtype=torch.float32, device=dev)
    off = torch.zeros((big.shape[0] + 1,), dtype=torch.int32, device=dev)
    with pytest.raises(nif.NifError) as e:
        nif.nif_segments_noalloc(h.h, [(0, 0, 0)], big, off, torch.zeros((1, 4), dtype=torch.int32, device=dev))
    assert e.value.status == nif.NIF_ERR_ARG and "NIF_NOALLOC_MAX_RAYS" in str(e.value)
    h.close()
