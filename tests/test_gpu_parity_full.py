"""Element-wise parity with the FP64 oracle at the training workload's sizes
(64^3 ellipsoid union, L = 16 levels, T = 2^19 rows per level, P = 9 gamma
terms, MLP 576-64-64-64-16, 2^18 segments per step).

At these sizes the CUDA path takes the branches the benchmark times: the
64 MiB FP32 tables put the encoder's distinct end points in rest-space order
(Morton counting sort), a segment's entry point that repeats the previous
exit point is encoded once and written to both rows, the backward walks the
distinct points in that order with its run-length cell cache, and the
split-TF32 MLP runs persistent CTAs over many 128-row jobs with the layer-0
weight gradient split over row ranges.

Inputs are seeded and synthetic (`synth.chained_segments`: straight lines
cut into consecutive pieces that share end points bit for bit, like the
segments of a training batch). Both sides take the same float32 inputs;
cells and ReLU branches are compared only where FP32 and FP64 must agree
(`tests/bounds.py`), and every float is compared element by element against
a bound derived from the FP32 arithmetic.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2604_24666_gb300 import synth as S
from tests import bounds as B

pytestmark = pytest.mark.gpu

NET = S.WORKLOADS["ellipsoids64_train"]["net"]


@pytest.fixture(scope="module")
def nif():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_24666_gb300 import nif as N
    N.lib()
    return N


@pytest.fixture(scope="module")
def handle(nif):
    h = nif.Nif(NET, S.ellipsoid_union_mesh())
    yield h
    h.close()


@pytest.fixture(scope="module")
def batch():
    """>= 2^14 segments whose every cell is certain, chained like a batch."""
    lin, _ = S.chained_segments(26000, seed=201, voxel_res=NET.voxel_res, gap=0.3)
    keep = B.certain_cells(NET, lin[:, 0:3]) & B.certain_cells(NET, lin[:, 3:6])
    lin = lin[keep]
    assert len(lin) >= 1 << 14
    tables = np.random.default_rng(202).uniform(-1, 1, (NET.levels, 1 << NET.log2_table, NET.feats)).astype(np.float32)
    return lin, tables


def _dev():
    return torch.device("cuda:0")


def test_encode_forward_sorted_dedup_matches_oracle(nif, handle, batch):
    lin, tables = batch
    net = NET
    handle.set_params(tables, S.init_params(net)[1])
    # the structure the deduplicating path exploits: most entry points repeat an exit point
    rep = (lin[1:, 0:3] == lin[:-1, 3:6]).all(1).mean()
    assert rep > 0.3, rep
    feats = nif.nif_encode_segments(handle.h, torch.from_numpy(lin).to(_dev()), net.in_dim).cpu().numpy()
    p0, p1 = lin[:, 0:3].astype(np.float64), lin[:, 3:6].astype(np.float64)
    ref = O.encode_segments(net, tables, p0, p1)
    bnd = np.concatenate([B.feature_bound(net, tables, p0), B.feature_bound(net, tables, p1)], 1)
    err = np.abs(feats - ref)
    assert np.all(err <= bnd), (err / bnd).max()
    # rows written twice: a repeated entry point's features equal the previous exit point's bit for bit
    half = net.in_dim // 2
    same = np.nonzero((lin[1:, 0:3] == lin[:-1, 3:6]).all(1))[0]
    assert np.array_equal(feats[same + 1, :half], feats[same, half:])


@pytest.mark.parametrize("out", ["bf16", "fp16"])
def test_encode_forward_fp16_tables_matches_oracle(nif, handle, batch, out):
    """The mixed path's encoder: FP16 table copy (32 MiB, sorted order too),
    16-bit feature rows. The oracle encodes with the tables rounded to FP16;
    the bound adds the rounding of each output to 16 bits."""
    lin, tables = batch
    net = NET
    handle.set_params(tables, S.init_params(net)[1])
    odt = nif.NIF_BF16 if out == "bf16" else nif.NIF_FP16
    feats = nif.nif_encode_segments(handle.h, torch.from_numpy(lin).to(_dev()), net.in_dim, out_dtype=odt,
                                    table_dtype=nif.NIF_FP16).float().cpu().numpy()
    t16 = tables.astype(np.float16).astype(np.float64)
    p0, p1 = lin[:, 0:3].astype(np.float64), lin[:, 3:6].astype(np.float64)
    ref = O.encode_segments(net, t16, p0, p1)
    bnd = np.concatenate([B.feature_bound(net, t16, p0), B.feature_bound(net, t16, p1)], 1)
    ulp = 2.0 ** -8 if out == "bf16" else 2.0 ** -11          # half an ulp, relative
    sub = 0.0 if out == "bf16" else 2.0 ** -25                 # half the FP16 subnormal spacing
    err = np.abs(feats - ref)
    tol = bnd * (1 + ulp) + ulp * np.abs(ref) + sub
    assert np.all(err <= tol), (err / tol).max()


_REF = {}


@pytest.mark.parametrize("split", [1, 2], ids=["levels-together", "level-halves"])
@pytest.mark.parametrize("det", [0, 1], ids=["l2-reductions", "deterministic"])
def test_encode_backward_sorted_matches_oracle(nif, handle, batch, det, split):
    """The table gradient at the training sizes; with NIF_KNOB_DETERMINISTIC
    the 64-bit fixed-point sums instead, whose bound adds 2^-(S+1) per
    contribution and whose second run must repeat the first bit for bit;
    with NIF_KNOB_BWD_SPLIT = 2 each task of the walk holds half of the
    levels."""
    lin, tables = batch
    net = NET
    handle.set_params(tables, S.init_params(net)[1])
    n = len(lin)
    df = np.random.default_rng(203).normal(size=(n, net.in_dim)).astype(np.float32)
    lint, dft = torch.from_numpy(lin).to(_dev()), torch.from_numpy(df).to(_dev())
    dtab = torch.zeros((net.levels, 1 << net.log2_table, net.feats), dtype=torch.float32, device=_dev())
    nif.nif_set_knob(handle.h, nif.NIF_KNOB_DETERMINISTIC, det)
    nif.nif_set_knob(handle.h, nif.NIF_KNOB_BWD_SPLIT, split)
    try:
        nif.nif_encode_segments_backward(handle.h, lint, dft, dtab)
        if det:
            again = torch.zeros_like(dtab)
            nif.nif_encode_segments_backward(handle.h, lint, dft, again)
            assert torch.equal(again, dtab)
    finally:
        nif.nif_set_knob(handle.h, nif.NIF_KNOB_DETERMINISTIC, 0)
        nif.nif_set_knob(handle.h, nif.NIF_KNOB_BWD_SPLIT, 0)
    g = dtab.cpu().numpy()
    half = net.in_dim // 2
    p = np.concatenate([lin[:, 0:3], lin[:, 3:6]]).astype(np.float64)
    d = np.concatenate([df[:, :half], df[:, half:]]).astype(np.float64)
    if "ref" not in _REF:
        _REF["ref"] = O.encode_points_backward(net, tables, p, d)[0]
    ref = _REF["ref"]
    key = ("bnd", det)
    if key not in _REF:
        _REF[key] = B.table_grad_bound(net, tables, p, d, fix_S=B.fixed_scale(n, net.n_terms, df) if det else None)
    bnd = _REF[key]
    err = np.abs(g - ref)
    assert np.all(err <= bnd), ((err / np.maximum(bnd, 1e-300)).max(), int((err > bnd).sum()))
    # untouched rows stay exactly zero
    assert np.all(g[ref == 0] == 0)
    # per level, relative L2 against the bar derived in tests/bounds.py
    for l in range(net.levels):
        rel = np.linalg.norm(g[l] - ref[l]) / np.linalg.norm(ref[l])
        assert rel <= B.rel_l2_bar(net, l), (l, rel)


def test_mlp_split_tf32_full_batch_matches_oracle(nif, handle):
    """Forward, dX and dW of the FP32 MLP at 2^18 rows: persistent CTAs take
    many 128-row jobs; the layer-0 weight gradient is split over row ranges.
    The forward runs twice, in per-layer launches and in one launch
    (NIF_KNOB_FP32_FUSED). Rows whose ReLU decisions FP32 could flip are left
    out before either side runs."""
    net = NET
    _, ws, s = S.init_params(net, seed=211)
    handle.set_params(S.init_params(net)[0], ws, s)
    n = 1 << 18
    rng = np.random.default_rng(212)
    x = rng.normal(size=(n + (n >> 3), net.in_dim)).astype(np.float32)
    x = x[B.relu_certain_rows(ws, x)][:n]
    assert len(x) == n
    xt = torch.from_numpy(x).to(_dev())
    ref, racts = O.mlp_forward(ws, x.astype(np.float64))
    for fused in (1, 0):
        nif.nif_set_knob(handle.h, nif.NIF_KNOB_FP32_FUSED, fused)
        acts = torch.zeros((net.mlp_depth, n, net.mlp_width), dtype=torch.float32, device=_dev())
        out = nif.nif_mlp_forward(handle.h, xt, acts=acts).cpu().numpy()
        # FP32 accumulation over K <= 576 terms (split TF32: each product to ~2^-21)
        np.testing.assert_allclose(out, ref, atol=2e-5 * np.abs(ref).max(), rtol=0)
        a = acts.cpu().numpy()
        for l in range(net.mlp_depth):
            np.testing.assert_allclose(a[l], racts[l + 1], atol=2e-5 * np.abs(racts[l + 1]).max(), rtol=0)
        del a
    dout = rng.normal(size=(n, 16)).astype(np.float32)
    dout[:, net.out_dim:] = 0
    nif.nif_zero_grad(handle.h)
    dx = nif.nif_mlp_backward(handle.h, xt, acts, torch.from_numpy(dout).to(_dev())).cpu().numpy()
    torch.cuda.synchronize()
    rdw, rdx = O.mlp_backward(ws, racts, dout.astype(np.float64))
    np.testing.assert_allclose(dx, rdx, atol=2e-5 * np.abs(rdx).max(), rtol=0)
    _, gws, _ = handle.get_grads()
    # dW_l = dY_l^T X_l over 2^18 rows: FP32 sums in TMEM per CTA, then one
    # atomic add per CTA. Bound: 2^-21 per split-TF32 product plus a sum of
    # R terms in FP32, both relative to the absolute sum |dY|^T |X|.
    g = dout.astype(np.float64)
    for i in range(len(ws) - 1, -1, -1):
        sabs = np.abs(g).T @ np.abs(racts[i])
        tol = (2.0 ** -21 + 2.0 ** -17) * sabs + 1e-6 * np.abs(rdw[i]).max()
        err = np.abs(gws[i] - rdw[i])
        assert np.all(err <= tol), (i, (err / tol).max())
        g = g @ np.asarray(ws[i], np.float64)
        if i > 0:
            g = g * (racts[i] > 0)
    # deterministic mode: each row range's sum stored and the ranges added in
    # order; the same bound, and a second run repeats the first bit for bit
    nif.nif_set_knob(handle.h, nif.NIF_KNOB_DETERMINISTIC, 1)
    try:
        runs = []
        for _ in range(2):
            nif.nif_zero_grad(handle.h)
            nif.nif_mlp_backward(handle.h, xt, acts, torch.from_numpy(dout).to(_dev()), want_dx=False)
            torch.cuda.synchronize()
            runs.append(handle.get_grads()[1])
    finally:
        nif.nif_set_knob(handle.h, nif.NIF_KNOB_DETERMINISTIC, 0)
    assert all(np.array_equal(a, b) for a, b in zip(runs[0], runs[1]))
    g = dout.astype(np.float64)
    for i in range(len(ws) - 1, -1, -1):
        sabs = np.abs(g).T @ np.abs(racts[i])
        tol = (2.0 ** -21 + 2.0 ** -17) * sabs + 1e-6 * np.abs(rdw[i]).max()
        err = np.abs(runs[0][i] - rdw[i])
        assert np.all(err <= tol), (i, (err / tol).max())
        g = g @ np.asarray(ws[i], np.float64)
        if i > 0:
            g = g * (racts[i] > 0)
