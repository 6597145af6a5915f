"""Helpers shared by the GPU parity tests (inputs and oracle filters only)."""
import numpy as np

import oracle as O
from paper_2604_24666_gb300 import synth as S

# A ray is compared bit-exactly when every decision it meets in the FP64
# oracle has at least this margin (world units): FP32 corner positions are
# good to ~5e-7, so 1e-5 leaves a factor of 20.
SEG_MARGIN = 1e-5
# A segment's label is compared exactly when the rest segment passes at
# least this far from every triangle edge / end (world units).
LABEL_MARGIN = 1e-5


def certain_rays(N, mesh, pose, rays, with_labels=False):
    """Indices of rays whose segment list (and labels) are decided with margin."""
    occ, ptr, idx = O.voxelize(N, mesh)
    seg = O.segments(N, occ, pose, rays)
    ok = seg.margin > SEG_MARGIN
    if with_labels and len(seg):
        p0, p1, _, _ = O.linearize(pose, rays, seg)
        lab = O.labels(mesh, ptr, idx, seg.vox, p0, p1)
        bad = np.zeros(len(rays), bool)
        np.logical_or.at(bad, seg.ray, lab["margin"] < LABEL_MARGIN)
        ok &= ~bad
    return np.nonzero(ok)[0]


def split_seg(off, segs_np):
    """Per-ray lists from the GPU's CSR (offsets, structured segments)."""
    return [segs_np[off[r]:off[r + 1]] for r in range(len(off) - 1)]


def random_tables(net, seed, scale=1.0):
    T = 1 << net.log2_table
    return np.random.default_rng(seed).uniform(-scale, scale, (net.levels, T, net.feats)).astype(np.float32)


def occupancy_biased_weights(net, seed):
    """Initial weights with the occupancy logit scaled up so queries hit."""
    _, ws, s = S.init_params(net, seed=seed)
    ws[-1][0, :] *= 4.0
    return ws, s


def evaluate_hits(mesh, pose, rays_np, hit, D, nrm, alb, mat):
    """Errors of predicted first hits against the exact deformed-mesh hits:
    hit IoU, distance MAE, mean normal angle (degrees), albedo L1 and
    material accuracy over rays where both hit."""
    t, tri = O.exact_hits(mesh, pose, rays_np)
    gt = np.isfinite(t)
    both = hit & gt
    dv = O.deform(pose, mesh.verts.astype(np.float64))
    tv = dv[mesh.tris[tri[both]]]
    gn = np.cross(tv[:, 1] - tv[:, 0], tv[:, 2] - tv[:, 0])
    gn /= np.linalg.norm(gn, axis=1, keepdims=True)
    c = np.clip((nrm[both] * gn).sum(1), -1, 1)
    return dict(iou=both.sum() / max(1, (hit | gt).sum()), dist=float(np.abs(D[both] - t[both]).mean()),
                normal=float(np.degrees(np.arccos(c)).mean()),
                albedo=float(np.abs(alb[both] - mesh.albedo[tri[both]]).mean()),
                material=float((mat[both] == mesh.material[tri[both]]).mean()))
