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


def test_segments_noalloc_counts_and_instances(nif):
    from paper_2604_24666_gb300 import synth as S
    dev = torch.device("cuda:0")
    mesh = S.torus_mesh()
    # a fresh handle holds buffers for one instance: more are refused, not allocated
    fresh = nif.Nif(S.NetConfig(voxel_res=16), mesh)
    rays = torch.from_numpy(S.sphere_rays(300, seed=5)).to(dev)
    inst = torch.tensor([0, 100, 200, 300], dtype=torch.int32, device=dev)
    off = torch.zeros((301,), dtype=torch.int32, device=dev)
    with pytest.raises(nif.NifError) as e:
        nif.nif_segments_noalloc(fresh.h, S.poses(3, seed=6), rays, off, None, inst_offsets=inst)
    assert e.value.status == nif.NIF_ERR_ARG
    fresh.close()

    h = nif.Nif(S.NetConfig(voxel_res=16), mesh)
    counts = [700, 0, 1234]
    n = sum(counts)
    inst = torch.from_numpy(np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)).to(dev)
    rays = torch.from_numpy(S.sphere_rays(n, seed=7)).to(dev)
    poses = S.poses(3, seed=8)
    ref_off, ref_segs = nif.nif_segments(h.h, poses, rays, inst_offsets=inst)   # sizes the handle for 3
    for call in range(2):
        # counts only (no segment rows): offsets and total as the allocating call gives them
        off = torch.full((n + 1,), -1, dtype=torch.int32, device=dev)
        total = nif.nif_segments_noalloc(h.h, poses, rays, off, None, inst_offsets=inst)
        torch.cuda.synchronize()
        assert total == ref_segs.shape[0] > 0, call
        assert torch.equal(off, ref_off), call
        # with rows
        segs = torch.full((total, 4), -1, dtype=torch.int32, device=dev)
        off2 = torch.full((n + 1,), -1, dtype=torch.int32, device=dev)
        assert nif.nif_segments_noalloc(h.h, poses, rays, off2, segs, inst_offsets=inst) == total
        torch.cuda.synchronize()
        assert torch.equal(off2, ref_off) and torch.equal(segs, ref_segs), call
    h.close()
