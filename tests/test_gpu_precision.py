"""Per-output error of the FP32 / BF16 / FP16 query paths against the FP64
oracle on a trained network: the config-1 torus network (L = 8, T = 2^14,
MLP 288-32-32-16), trained on the GPU in FP32 at 16^3 voxels (4000 steps of
2^16 segments over poses U[-1,1]^3), queried on the 16^3 grid and on the
128^3 grid of the precision workload (same encoding and MLP; a network
trained at 128^3 predicts no hit, its finest level having 68 cells per axis).

Stated bounds (asserted; the measured values are printed):
  FP32:      hit IoU >= 0.999, same first-hit segment on >= 99.9 % of the
             rays both hit, |D| p99 <= 1e-3, normal p99 <= 1 deg, albedo
             p99 <= 1e-3, material >= 99.5 %;
  BF16/FP16: hit IoU >= 0.99, same first-hit segment >= 98 %, |D| p99 <=
             5e-3, normal p99 <= 5 deg, albedo p99 <= 5e-2, material >= 98 %.
Distance, normal, albedo and material are compared where the first hit is
in the same segment (|dD| < half a voxel); a decision flipped on an earlier
segment moves the hit by about a voxel and is counted by the second bound.
The oracle takes its own segments in FP64 (rays whose decision margin is too
small for FP32 are left out, as in the segment parity tests).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2604_24666_gb300 import synth as S
from tests.gpu_common import certain_rays

pytestmark = pytest.mark.gpu


def _fields(nif, hits):
    a = hits.cpu().numpy().view(nif.HIT_DTYPE).reshape(-1)
    return (a["hit"] > 0, a["D"].astype(np.float64), a["n"].astype(np.float64), a["albedo"].astype(np.float64),
            a["material"])


def _errs(ref, got, N):
    """Hit IoU; among rays both sides hit, the fraction whose first hit lies
    in the same segment (|dD| below half a voxel, 1/(2N): a flipped decision
    on an earlier segment moves the hit by about a voxel, an event counted
    like a hit flip, not as a distance error); and over those rays the
    distance, normal, albedo and material errors."""
    h0, d0, n0, a0, m0 = ref
    h1, d1, n1, a1, m1 = got
    both = h0 & h1
    same = both.copy()
    same[both] = np.abs(d0[both] - d1[both]) < 0.5 / N
    ang = np.degrees(np.arccos(np.clip((n0[same] * n1[same]).sum(1), -1, 1)))
    return dict(iou=both.sum() / max(1, (h0 | h1).sum()), same=same.sum() / max(1, both.sum()),
                d99=np.percentile(np.abs(d0[same] - d1[same]), 99), n99=np.percentile(ang, 99),
                a99=np.percentile(np.abs(a0[same] - a1[same]).max(1), 99), mat=(m0[same] == m1[same]).mean())


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_24666_gb300 import nif
    w = S.WORKLOADS["torus16_fwd"]
    h = nif.Nif(w["net"], S.make_mesh(w["shape"]), precision=nif.NIF_FP32, seed=51)
    for step in range(4000):
        nif.nif_train_step(h.h, 1 << 16, 16, 5000 + step, lr_grid=1e-2, lr_mlp=5e-3, want_loss=False)
    params = h.get_params()
    h.close()
    return params


@pytest.mark.parametrize("workload", ["torus16_fwd", "torus128_query"])
def test_query_precision_against_fp64_oracle(trained, workload):
    from paper_2604_24666_gb300 import nif
    w = S.WORKLOADS[workload]
    net = w["net"]
    mesh = S.make_mesh(w["shape"])
    tables, ws, s = trained
    hs = {}
    for name, p in (("fp32", nif.NIF_FP32), ("bf16", nif.NIF_BF16), ("fp16", nif.NIF_FP16)):
        hs[name] = nif.Nif(net, mesh, precision=p, seed=51)
        hs[name].set_params(tables, ws, s)
    pose = S.poses(1, seed=52)[0]
    rays_np = S.sphere_rays(3000, seed=54)
    rays_np = rays_np[certain_rays(net.voxel_res, mesh, pose, rays_np)]
    rays = torch.from_numpy(rays_np).cuda()
    occ, _, _ = O.voxelize(net.voxel_res, mesh)
    seg = O.segments(net.voxel_res, occ, pose, rays_np)
    p0, p1, ld, lr = O.linearize(pose, rays_np, seg)
    out = O.mlp_forward([x.astype(np.float64) for x in ws], O.encode_segments(net, tables, p0, p1))[0]
    res = O.reconstruct(net, pose, rays_np, seg, out, p0, p1, ld, lr)
    ref = (res["hit"] > 0, res["D"], res["normal"], res["albedo"], res["material"])
    table = {}
    for name, hh in hs.items():
        table[name] = _errs(ref, _fields(nif, nif.nif_query(hh.h, [pose], rays)), net.voxel_res)
        hh.close()
    print(workload, "per-output error vs FP64 oracle:",
          {k: {m: float(v) for m, v in e.items()} for k, e in table.items()}, "oracle hits:", int(ref[0].sum()))
    assert ref[0].sum() > 100
    e = table["fp32"]
    assert e["iou"] >= 0.999 and e["same"] >= 0.999
    assert e["d99"] <= 1e-3 and e["n99"] <= 1.0 and e["a99"] <= 1e-3 and e["mat"] >= 0.995
    for name in ("bf16", "fp16"):
        e = table[name]
        assert e["iou"] >= 0.99 and e["same"] >= 0.98, name
        assert e["d99"] <= 5e-3 and e["n99"] <= 5.0 and e["a99"] <= 5e-2 and e["mat"] >= 0.98, name
