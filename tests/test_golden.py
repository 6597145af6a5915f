"""Stored values: the paper's Table 1 (cited in the file) and the FP64 oracle's
outputs for a small fixed case, written by tests/golden/make_oracle_golden.py.
The oracle must still reproduce its stored values: a change to its
arithmetic shows up here and has to name the passage that justifies it."""
import json
import os

import numpy as np

import oracle as O
from paper_2604_24666_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_table1():
    rows = {}
    for line in open(os.path.join(GOLDEN, "table1.txt")):
        if line.strip() and not line.startswith("#"):
            m, d, n = line.split()
            rows[m] = (float(d), float(n))
    return rows


def test_table1_fixture():
    t = load_table1()
    assert set(t) == {"LSNIF", "Deformed", "Proposed"}
    # the paper ranks the proposed method first in both metrics
    assert min(t, key=lambda k: t[k][0]) == "Proposed" and min(t, key=lambda k: t[k][1]) == "Proposed"


def test_oracle_reproduces_stored_case():
    g = json.load(open(os.path.join(GOLDEN, "oracle_torus16.json")))
    net = S.NetConfig()
    mesh = S.torus_mesh()
    N = g["voxel_res"]
    occ, ptr, idx = O.voxelize(N, mesh)
    rays = np.asarray(g["rays"], np.float32)
    seg = O.segments(N, occ, tuple(g["pose"]), rays)
    np.testing.assert_array_equal(seg.count, g["count"])
    np.testing.assert_array_equal(seg.vox, g["voxel"])
    np.testing.assert_allclose(seg.t0, g["t0"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(seg.t1, g["t1"], rtol=1e-12, atol=1e-14)
    p0, p1, _, l_rest = O.linearize(tuple(g["pose"]), rays, seg)
    np.testing.assert_allclose(p0, g["p0"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(p1, g["p1"], rtol=1e-12, atol=1e-14)
    tables, ws, s = S.init_params(net, seed=5)
    x = O.encode_segments(net, tables, p0, p1)
    np.testing.assert_allclose(x[0], g["features_first_segment"], rtol=1e-12, atol=1e-15)
    lab = O.labels(mesh, ptr, idx, seg.vox, p0, p1)
    out, _ = O.mlp_forward(ws, x)
    np.testing.assert_allclose(out[0], g["mlp_out_first_segment"], rtol=1e-12, atol=1e-15)
    tot, _, _, _ = O.loss(net, out, lab, s, l_rest)
    assert abs(tot - g["loss_total"]) <= 1e-12 * abs(g["loss_total"])
