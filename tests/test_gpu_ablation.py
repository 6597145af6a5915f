"""Paper-setting ablation (Sec. 3.1, Table 1; Sec. 3.2 comparison settings).

Three networks on the ellipsoid union at 32^3 voxels with a two-level grid of
base resolution 64 (F_d = 2 here; the paper uses 3, which this library does
not build), 3000 GPU training steps of 2^16 segments each:
  proposed     F = 3 positional bands, uncertainty-weighted losses, ReLU head
               with log-space distance error (Sec. 2.3, 2.4);
  deformed     the "Deformed" baseline: no positional encoding, fixed task
               weights, sigmoid distance head with a plain squared error,
               trained on the same pose distribution;
  lsnif        the same ablated settings trained on the static pose only
               (the original single-pose LSNIF protocol).
All are evaluated on the static (identity) pose against the exact first hit
of the mesh, as in Table 1. The paper's claim checked here: the proposed
method has the lowest distance and normal error.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2604_24666_gb300 import synth as S
from tests.gpu_common import evaluate_hits

pytestmark = pytest.mark.gpu


def test_proposed_beats_deformed_baseline_and_single_pose_lsnif():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_24666_gb300 import nif
    mesh = S.ellipsoid_union_mesh()
    base = dict(voxel_res=32, levels=2, feats=2, log2_table=19, base_res=64, growth=1.5, mlp_depth=2,
                mlp_width=64, n_materials=4)
    ablated = nif.NIF_FLAG_FIXED_TASK_WEIGHTS | nif.NIF_FLAG_SIGMOID_DISTANCE
    variants = {"proposed": (S.NetConfig(pe_bands=3, **base), 0, True),
                "deformed": (S.NetConfig(pe_bands=0, **base), ablated, True),
                "lsnif": (S.NetConfig(pe_bands=0, **base), ablated, False)}
    rays_np = S.sphere_rays(3000, seed=4343)
    rays = torch.from_numpy(rays_np).cuda()
    table = {}
    for name, (net, flags, posed) in variants.items():
        h = nif.Nif(net, mesh, seed=11, flags=flags)
        for step in range(3000):
            if posed:
                nif.nif_train_step(h.h, 1 << 16, 16, 9000 + step, lr_grid=1e-2, lr_mlp=5e-3, want_loss=False)
            else:
                r = nif.nif_sample_rays(h.h, 9000 + step, 0, 40000)
                nif.nif_train_step_rays(h.h, [(0.0, 0.0, 0.0)], r, 1 << 16, lr_grid=1e-2, lr_mlp=5e-3,
                                        want_loss=False)
        pose = np.zeros(3, np.float32)
        hq = nif.nif_query(h.h, [pose], rays).cpu().numpy().view(nif.HIT_DTYPE).reshape(-1)
        table[name] = evaluate_hits(mesh, pose, rays_np, hq["hit"] > 0, hq["D"].astype(np.float64),
                                    hq["n"].astype(np.float64), hq["albedo"], hq["material"])
        h.close()
    print("static-pose errors (distance MAE, normal deg):",
          {k: (round(v["dist"], 5), round(v["normal"], 2)) for k, v in table.items()})
    # the method the paper's Table 1 (tests/golden/table1.txt) ranks first in
    # each metric must rank first here too
    from tests.test_golden import load_table1
    paper = load_table1()
    names = {"Proposed": "proposed", "Deformed": "deformed", "LSNIF": "lsnif"}
    for col, key in ((0, "dist"), (1, "normal")):
        best = names[min(paper, key=lambda m: paper[m][col])]
        for other in table:
            if other != best:
                assert table[best][key] < table[other][key], (key, best, other)
