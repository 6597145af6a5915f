"""Writes oracle_torus16.json: the FP64 oracle's outputs for a small fixed case
(16^3 torus, one pose, a few rays whose voxel and label decisions hold with
margin), so that a
later change to the oracle's arithmetic shows up as a difference to a stored
value. Calls only oracle/ and the seeded input generators.

    python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2604_24666_gb300 import synth as S  # noqa: E402

POSE = (0.4, -0.7, 0.3)
N = 16


def case():
    net = S.NetConfig()
    mesh = S.torus_mesh()
    occ, ptr, idx = O.voxelize(N, mesh)
    rays = S.sphere_rays(400, seed=71)
    seg = O.segments(N, occ, POSE, rays)
    q0, q1, _, _ = O.linearize(POSE, rays, seg)
    lab_margin = O.labels(mesh, ptr, idx, seg.vox, q0, q1)["margin"]
    # rays whose voxel decisions and label decisions all hold with margin
    keep = [r for r in range(len(rays))
            if seg.margin[r] > 1e-4 and seg.count[r] >= 2 and lab_margin[seg.off[r]:seg.off[r + 1]].min() > 1e-4][:6]
    rays = rays[keep]
    seg = O.segments(N, occ, POSE, rays)
    p0, p1, l_def, l_rest = O.linearize(POSE, rays, seg)
    tables, ws, s = S.init_params(net, seed=5)
    x = O.encode_segments(net, tables, p0, p1)
    lab = O.labels(mesh, ptr, idx, seg.vox, p0, p1)
    out, _ = O.mlp_forward(ws, x)
    tot, parts, _, _ = O.loss(net, out, lab, s, l_rest)
    return {
        "pose": list(POSE), "voxel_res": N, "rays": rays.tolist(),
        "count": seg.count.tolist(), "voxel": seg.vox.tolist(),
        "t0": seg.t0.tolist(), "t1": seg.t1.tolist(),
        "p0": p0.tolist(), "p1": p1.tolist(),
        "features_first_segment": x[0].tolist(),
        "mlp_out_first_segment": out[0].tolist(),
        "loss_total": float(tot),
    }


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_torus16.json")
    with open(path, "w") as f:
        json.dump(case(), f, indent=1)
    print("wrote", path)
