"""The CUDA path through the C ABI against the oracle's stored values for the
small fixed case of tests/golden/oracle_torus16.json (rays whose voxel and
label decisions hold with a margin above 1e-4, so every decision is certain)."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2604_24666_gb300 import synth as S

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_cuda_path_matches_stored_oracle_case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_24666_gb300 import nif
    g = json.load(open(os.path.join(GOLDEN, "oracle_torus16.json")))
    net = S.NetConfig()
    h = nif.Nif(net, S.torus_mesh())
    tables, ws, s = S.init_params(net, seed=5)
    h.set_params(tables, ws, s)
    pose = tuple(g["pose"])
    rays = torch.from_numpy(np.asarray(g["rays"], np.float32)).cuda()
    offs, segs = nif.nif_segments(h.h, [pose], rays)
    sg = segs.cpu().numpy().view(nif.SEGMENT_DTYPE).reshape(-1)
    np.testing.assert_array_equal(np.diff(offs.cpu().numpy().astype(np.int64)), g["count"])
    np.testing.assert_array_equal(sg["voxel"], g["voxel"])
    # FP32 corners and hull tests against FP64 (distances of order 1)
    np.testing.assert_allclose(sg["t0"], g["t0"], atol=1e-5)
    np.testing.assert_allclose(sg["t1"], g["t1"], atol=1e-5)
    lin = nif.nif_linearize(h.h, [pose], rays, segs)
    ln = lin.cpu().numpy().reshape(-1, 8)
    np.testing.assert_allclose(ln[:, 0:3], g["p0"], atol=1e-5)
    np.testing.assert_allclose(ln[:, 3:6], g["p1"], atol=1e-5)
    lab = nif.nif_labels(h.h, segs, lin)
    feat = nif.nif_encode_segments(h.h, lin, net.in_dim)
    # the FP32 encoder at the GPU's own end points (FP32 trilinear sums of small table values)
    f0 = feat[0].cpu().numpy()
    np.testing.assert_allclose(f0, g["features_first_segment"], atol=1e-5 * max(1.0, np.abs(tables).max()))
    out = nif.nif_mlp_forward(h.h, feat)
    np.testing.assert_allclose(out[0].cpu().numpy(), g["mlp_out_first_segment"], rtol=1e-3, atol=1e-5)
    parts, _ = nif.nif_loss(h.h, out, lab, lin)
    assert abs(parts[0] - g["loss_total"]) <= 1e-3 * abs(g["loss_total"]), (parts[0], g["loss_total"])
    h.close()
