"""Per-element error bounds for comparing the FP32 CUDA path with the FP64
oracle on identical inputs (test infrastructure).

The bounds follow from the arithmetic of the hash-grid encoding (Sec. 2.3,
Eq. 1) and are evaluated with the oracle's own helpers (`_cell`,
`grid_index`, `gamma`, `level_res`); nothing here reads a GPU result.

Notation: u = 2^-24 (FP32 unit roundoff); a point's grid coordinate is u_t
for term t of gamma; level l has N_l cells. Two error sources:

* rounding: the kernels form the trilinear weights (3 factors), products
  and sums in FP32;
* the sin/cos terms: the kernel's u = (sincosf(2^k p) + 1)/2 differs from
  the oracle's FP64 value by at most DU (CUDA's sincosf is within 2 ulp,
  plus the FP32 rounding of the sum). At a fixed cell a weight factor moves
  by N_l * DU, so a trilinear weight moves by at most 3 N_l DU.

Cells are only compared where they are unique: `certain_cells` rejects
points whose sin/cos-term coordinates at any level lie within CELL_MARGIN *
N_l * DU of a cell face. The two sides' q = u N_l differ by at most
N_l (DU + 2^-23) (the oracle rounds its u and the product to FP32 as the
kernel does), below that margin. The x term's u is the same FP32 value on
both sides, so its cells agree exactly.

Relative L2 of a table gradient per level: FP32 summation over k terms
grows like sqrt(k) u, far below 1e-4; the sin/cos weights add about
3 N_l DU_TYP relative (DU_TYP = 6e-8, one FP32 ulp of u near 1, is the size
of a typical sincosf difference), which passes 1e-4 at the finest levels
(N_l up to 1751 at L = 16), so the per-level bar is
1e-4 + 3 N_l DU_TYP (`rel_l2_bar`).
"""
from __future__ import annotations

import math

import numpy as np

import oracle as O

U32 = 2.0 ** -24
DU = 4e-7
CELL_MARGIN = 2.0


DU_TYP = 6e-8


def rel_l2_bar(net, l):
    return 1e-4 + 3 * O.level_res(net)[l] * DU_TYP


def certain_cells(net, p):
    """bool [n]: every sin/cos-term cell of p is decided with margin."""
    _, u = O.gamma(net, np.asarray(p, np.float64))
    ok = np.ones(len(u), bool)
    for t in range(1, u.shape[1]):
        for N in O.level_res(net):
            q = u[:, t] * N
            dist = np.abs(q - np.round(q)).min(axis=1)
            ok &= dist > CELL_MARGIN * N * DU
    return ok


def _terms(net, p):
    pc = np.asarray(p, np.float64)
    _, u = O.gamma(net, pc)
    return pc, u


def feature_bound(net, tables, p):
    """[n, P*L*F_d] bound on |psi_fp32(p) - psi(p)| (same cells):
    12 u sum_c w_c |t_c| + [sin/cos] 3 N_l DU sum_c |t_c|."""
    tables = np.asarray(tables, np.float64)
    _, u = _terms(net, p)
    n, P = u.shape[0], u.shape[1]
    res = O.level_res(net)
    out = np.zeros((n, P, net.levels, net.feats))
    for t in range(P):
        for l in range(net.levels):
            i0, w = O._cell(net, l, u[:, t])
            for c in O._CORNERS:
                idx = O.grid_index(net, l, i0 + c)
                wt = np.prod(np.where(c == 1, w, 1.0 - w), axis=1)
                a = np.abs(tables[l][idx])
                out[:, t, l, :] += 12 * U32 * wt[:, None] * a
                if t > 0:
                    out[:, t, l, :] += 3 * res[l] * DU * a
    return out.reshape(n, -1)


def loss_grad_bound(net, out, lab, s, l_rest, out_err, flags=0):
    """[S, O] first-order bound on how much the loss gradient dL/dout moves
    when each output column j moves by at most out_err[j]: rows are
    independent, so perturbing a whole column at once and differencing the
    oracle's own gradient gives sum_j |d(dL/dout)/d out_j| out_err[j] for
    every row."""
    out = np.asarray(out, np.float64)
    err = np.zeros_like(out)
    for j in range(out.shape[1]):
        if out_err[j] == 0:
            continue
        e = np.zeros(out.shape[1])
        e[j] = out_err[j]
        hi = O.loss(net, out + e, lab, s, l_rest, flags)[2]
        lo = O.loss(net, out - e, lab, s, l_rest, flags)[2]
        err += 0.5 * np.abs(hi - lo)
    return err


def fixed_scale(n_segments, P, dfeat):
    """Scale exponent S of the deterministic table gradient for a call on
    n_segments segments with gradients dfeat (float32, as the GPU holds
    them): every sum is bounded by B = 2 n P max|dfeat|, and S is the largest
    integer with B 2^S < 2^61, at most 100 (0 when B = 0). Computed in the same double
    arithmetic and order as the library, so both sides get the same S."""
    m = float(np.abs(np.asarray(dfeat, np.float32)).max()) if np.size(dfeat) else 0.0
    b = 2.0 * float(n_segments) * float(P) * m
    if b == 0.0:
        return 0
    s = 61 - math.frexp(b)[1]
    assert s >= -60, "gradients this large are reported as non-finite"
    return min(s, 100)


def table_grad_bound(net, tables, p, dfeat, dfeat_err=0.0, fix_S=None):
    """[L, T, F_d] bound on the FP32 table gradient of sum(dfeat * psi(p))
    against the oracle's (same cells). Entry e with contributions w_i d_i,
    i = 1..k_e:
        (k_e + 6) u sum w_i |d_i|          rounding of weights, products, sums
      + 3 N_l DU sum_{i sin/cos} |d_i|     sin/cos weights
      + sum w_i dfeat_err_i                error of the given gradients
    dfeat_err is a scalar or per element of dfeat. Several (p, dfeat) pairs
    are summed by calling this on the stacked arrays. fix_S (deterministic
    mode) adds k_e 2^-(S+1): each contribution rounded to a multiple of 2^-S."""
    tables = np.asarray(tables, np.float64)
    _, u = _terms(net, p)
    n, P = u.shape[0], u.shape[1]
    d = np.abs(np.asarray(dfeat, np.float64)).reshape(n, P, net.levels, net.feats)
    de = np.broadcast_to(np.asarray(dfeat_err, np.float64), (n, P * net.levels * net.feats))
    de = de.reshape(n, P, net.levels, net.feats)
    res = O.level_res(net)
    A = np.zeros_like(tables)
    B = np.zeros_like(tables)
    E = np.zeros_like(tables)
    K = np.zeros(tables.shape[:2])
    for t in range(P):
        for l in range(net.levels):
            i0, w = O._cell(net, l, u[:, t])
            for c in O._CORNERS:
                idx = O.grid_index(net, l, i0 + c)
                wt = np.prod(np.where(c == 1, w, 1.0 - w), axis=1)
                np.add.at(A[l], idx, wt[:, None] * d[:, t, l, :])
                np.add.at(K[l], idx, 1.0)
                np.add.at(E[l], idx, wt[:, None] * de[:, t, l, :])
                if t > 0:
                    np.add.at(B[l], idx, d[:, t, l, :])
    res_col = np.asarray(res, np.float64)[:, None, None]
    fix = 0.0 if fix_S is None else K[..., None] * 2.0 ** -(fix_S + 1)
    return (K[..., None] + 6) * U32 * A + 3 * res_col * DU * B + E + fix


def point_grad_bound(net, tables, p, dfeat, dfeat_err=0.0):
    """[n, 3] bound on the FP32 dL/dp of sum(dfeat * psi(p)) (same cells).
    A term of dp_a is s_c N_l others_{c,a} val_c chain_{t,a} with
    val_c = sum_f t_cf d_f, others the product of the two other weight
    factors and chain = du/dp (1, 2^(k-1) cos, -2^(k-1) sin):
        16 u sum |term|                                   rounding
      + [sin/cos] 2 N_l DU N_l |val| |chain|              others at moved u
      + [sin/cos] N_l others |val| 2^(k-1) 2.4e-7         sincosf in chain
      + dfeat_err N_l others |chain| sum_f |t_cf|         given gradients
    zero where p was clamped (both sides)."""
    tables = np.asarray(tables, np.float64)
    pc, u = _terms(net, p)
    inside = (pc >= 0.0) & (pc <= 1.0)
    pcl = np.clip(pc, 0.0, 1.0)
    n, P = u.shape[0], u.shape[1]
    d = np.asarray(dfeat, np.float64).reshape(n, P, net.levels, net.feats)
    res = O.level_res(net)
    chain = np.ones((n, P, 3))
    scale = np.ones(P)
    for k in range(net.pe_bands):
        f = 2.0 ** k
        chain[:, 1 + 2 * k] = np.abs(0.5 * f * np.cos(f * pcl))
        chain[:, 2 + 2 * k] = np.abs(0.5 * f * np.sin(f * pcl))
        scale[1 + 2 * k] = scale[2 + 2 * k] = 0.5 * f
    out = np.zeros((n, 3))
    for t in range(P):
        for l in range(net.levels):
            i0, w = O._cell(net, l, u[:, t])
            N = res[l]
            for c in O._CORNERS:
                idx = O.grid_index(net, l, i0 + c)
                tab = tables[l][idx]
                val = (np.abs(tab) * np.abs(d[:, t, l, :])).sum(1)     # >= |val_c|, covers its rounding
                tabs = np.abs(tab).sum(1)
                fw = np.where(c == 1, w, 1.0 - w)
                for a in range(3):
                    others = np.prod(np.delete(fw, a, axis=1), axis=1)
                    term = N * others * val * chain[:, t, a]
                    out[:, a] += 16 * U32 * term + dfeat_err * N * others * chain[:, t, a] * tabs
                    if t > 0:
                        out[:, a] += 2 * N * DU * N * val * chain[:, t, a] + N * others * val * scale[t] * 2.4e-7
    return np.where(inside, out, 0.0)


def relu_certain_rows(ws, x, margin=1e-4):
    """bool [n]: every hidden pre-activation of the FP64 MLP on x is at least
    margin * (its layer's largest |z|) away from 0, so FP32 and FP64 take the
    same ReLU branch."""
    h = np.asarray(x, np.float64)
    ok = np.ones(len(h), bool)
    for w in ws[:-1]:
        z = h @ np.asarray(w, np.float64).T
        ok &= np.abs(z).min(axis=1) > margin * np.abs(z).max()
        h = np.maximum(z, 0.0)
    return ok


def mlp_abs(ws, x):
    """Forward of |x| through |W| (the layers' absolute sums, ReLU-free):
    row-wise scales of the FP32 rounding of each output."""
    h = np.abs(np.asarray(x, np.float64))
    for w in ws:
        h = h @ np.abs(np.asarray(w, np.float64)).T
    return h
