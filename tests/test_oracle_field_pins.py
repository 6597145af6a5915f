"""Pins of the oracle's learned deformation field (our reading of the paper's
Sec. 4 future work: a rest-space displacement lattice, trilinear, composed
before the parameterised deformation, D(p) = D_theta(p + u(p))).

Each pin checks the oracle against something other than itself: finite
differences, closed forms for affine fields (which trilinear interpolation
reproduces exactly), translation invariance of the segment list, exact
agreement with the analytic deformation at the lattice nodes and its O(h^2)
convergence between them.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_24666_gb300 import synth as S


def _random_field(G, seed, lip=0.4):
    """Smooth random field scaled so that its Lipschitz bound is `lip`."""
    rng = np.random.default_rng(seed)
    f = rng.normal(size=(G, G, G, 3))
    return f * (lip / O.field_lipschitz(f))


def _affine_field(G, A, b):
    g = np.arange(G, dtype=np.float64) / (G - 1)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    x = np.stack([X, Y, Z], -1)
    return x @ np.asarray(A).T + np.asarray(b)


def test_zero_field_is_the_analytic_deformation():
    rng = np.random.default_rng(1)
    p = rng.uniform(0, 1, (500, 3))
    pose = (0.7, -0.9, 0.4)
    z = np.zeros((5, 5, 5, 3))
    np.testing.assert_array_equal(O.deform_field(pose, z, p), O.deform(pose, p))
    y = O.deform(pose, p)
    np.testing.assert_array_equal(O.inverse_field(pose, z, y), O.inverse(pose, y))
    np.testing.assert_allclose(O.jacobian_field(pose, z, p), O.jacobians(pose, p)[0], rtol=0, atol=1e-15)


def test_affine_field_closed_forms():
    """Trilinear interpolation reproduces an affine u(p) = A p + b exactly:
    du/dp = A, the Lipschitz bound is ||A||_F, and the inverse of the field
    alone is (I + A)^-1 (q - b)."""
    rng = np.random.default_rng(2)
    A = rng.normal(size=(3, 3)) * 0.1
    b = rng.normal(size=3) * 0.02
    f = _affine_field(4, A, b)
    p = rng.uniform(0, 1, (400, 3))
    np.testing.assert_allclose(O.field_displacement(f, p), p @ A.T + b, atol=1e-14)
    np.testing.assert_allclose(O.field_grad(f, p), np.broadcast_to(A, (400, 3, 3)), atol=1e-12)
    assert abs(O.field_lipschitz(f) - np.linalg.norm(A)) < 1e-12
    q = p + p @ A.T + b
    np.testing.assert_allclose(O.field_inverse(f, q), p, atol=1e-13)
    # closed form of the inverse where it stays inside the cube
    inv = np.linalg.solve(np.eye(3) + A, (q - b).T).T
    np.testing.assert_allclose(O.field_inverse(f, q), inv, atol=1e-13)


@pytest.mark.parametrize("pose", [(0.0, 0.0, 0.0), (0.8, -1.2, 0.6), (-1.0, 1.5, -1.0)])
def test_field_round_trip_and_error_bound(pose):
    f = _random_field(6, 3, lip=0.45)
    lip = O.field_lipschitz(f)
    assert lip < 1
    rng = np.random.default_rng(4)
    p = rng.uniform(-0.02, 1.02, (2000, 3))
    y = O.deform_field(pose, f, p)
    back = O.inverse_field(pose, f, y)
    np.testing.assert_allclose(back, p, atol=1e-12)
    # a posteriori bound: |p - p*| <= |F(p)| / (1 - l) for any p
    q = O.inverse(pose, y)
    trial = q - O.field_displacement(f, q)                    # one fixed-point step
    F = trial + O.field_displacement(f, trial) - q
    assert np.all(np.linalg.norm(trial - p, axis=1) <= np.linalg.norm(F, axis=1) / (1 - lip) + 1e-13)


def test_field_jacobians_match_finite_differences():
    f = _random_field(5, 5, lip=0.4)
    pose = (0.5, -0.7, 0.3)
    rng = np.random.default_rng(6)
    p = rng.uniform(0.03, 0.97, (300, 3))
    h = 1e-6
    J = O.jacobian_field(pose, f, p)
    G = O.field_grad(f, p)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (O.deform_field(pose, f, p + e) - O.deform_field(pose, f, p - e)) / (2 * h)
        fdu = (O.field_displacement(f, p + e) - O.field_displacement(f, p - e)) / (2 * h)
        # away from the lattice's cell faces the field is smooth
        ok = np.abs((p * 4) - np.round(p * 4)).min(axis=1) > 2 * h * 4
        np.testing.assert_allclose(J[ok, :, a], fd[ok], atol=1e-7)
        np.testing.assert_allclose(G[ok, :, a], fdu[ok], atol=1e-7)


def test_lipschitz_bound_holds():
    f = _random_field(7, 7, lip=0.8)
    rng = np.random.default_rng(8)
    p = rng.uniform(0, 1, (5000, 3))
    norms = np.linalg.norm(O.field_grad(f, p), ord=2, axis=(1, 2))
    assert norms.max() <= O.field_lipschitz(f) + 1e-12
    assert norms.max() > 0.3 * O.field_lipschitz(f)


def test_field_from_pose_agrees_at_nodes_and_converges():
    pose = (0.9, -1.3, 0.7)
    for G in (5, 9):
        f = O.field_from_pose(G, pose)
        g = np.arange(G) / (G - 1)
        Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
        nodes = np.stack([X, Y, Z], -1).reshape(-1, 3)
        np.testing.assert_allclose(O.deform_field((0, 0, 0), f, nodes), O.deform(pose, nodes), atol=1e-15)
    rng = np.random.default_rng(9)
    p = rng.uniform(0, 1, (4000, 3))
    err = [np.abs(O.deform_field((0, 0, 0), O.field_from_pose(G, pose), p) - O.deform(pose, p)).max()
           for G in (5, 9, 17)]
    # trilinear interpolation error: O(h^2), a factor about 4 per halving of h
    assert err[0] / err[1] > 3.0 and err[1] / err[2] > 3.0, err


def test_segments_follow_a_translating_field():
    """A constant field b moves every hull by b (zero pose): the segment list
    of a ray equals the list of the same ray moved by -b without a field, and
    a zero field changes nothing."""
    mesh = S.torus_mesh()
    N = 16
    occ, _, _ = O.voxelize(N, mesh)
    rays = S.sphere_rays(400, seed=10)
    b = np.array([0.013, -0.021, 0.008])
    f = np.broadcast_to(b, (3, 3, 3, 3)).copy()
    s1 = O.segments(N, occ, (0, 0, 0), rays, field=f)
    moved = rays.copy()
    moved[:, 0:3] -= b.astype(np.float32)
    s2 = O.segments(N, occ, (0, 0, 0), moved)
    ok = (s1.margin > 1e-6) & (s2.margin > 1e-6)
    for r in np.nonzero(ok)[0]:
        a1, b1 = s1.off[r], s1.off[r + 1]
        a2, b2 = s2.off[r], s2.off[r + 1]
        assert np.array_equal(s1.vox[a1:b1], s2.vox[a2:b2]), r
        np.testing.assert_allclose(s1.t0[a1:b1], s2.t0[a2:b2], atol=1e-6)
    pose = (0.4, -0.6, 0.2)
    z = np.zeros((3, 3, 3, 3))
    s3 = O.segments(N, occ, pose, rays, field=z)
    s4 = O.segments(N, occ, pose, rays)
    assert np.array_equal(s3.vox, s4.vox) and np.array_equal(s3.t0, s4.t0)


def test_field_gradient_matches_finite_differences():
    """d/d(delta) of sum(dfeat * psi(D^-1(x))) at fixed deformed points x,
    against central differences of the whole chain (inverse, encoding)."""
    net = S.NetConfig(levels=2, log2_table=6, pe_bands=1, base_res=2)
    rng = np.random.default_rng(11)
    tables = rng.uniform(-1, 1, (net.levels, 1 << net.log2_table, net.feats))
    G = 3
    f = _random_field(G, 12, lip=0.3)
    pose = (0.3, -0.5, 0.2)
    p0 = rng.uniform(0.1, 0.9, (24, 3))
    p1 = np.clip(p0 + rng.normal(0, 0.05, (24, 3)), 0.05, 0.95)
    x0, x1 = O.deform_field(pose, f, p0), O.deform_field(pose, f, p1)
    df = rng.normal(size=(24, net.in_dim))

    def objective(field):
        q0, q1 = O.inverse_field(pose, field, x0), O.inverse_field(pose, field, x1)
        return float((df * O.encode_segments(net, tables, q0, q1)).sum())

    g = O.field_gradient(net, tables, pose, f, O.inverse_field(pose, f, x0), O.inverse_field(pose, f, x1), df)
    # the oracle takes the hash-grid cell coordinate in FP32 (as the kernels
    # do), so its forward is quantised at ~1e-7: a larger step keeps the
    # quantisation error of the difference at ~1e-3 (the encoding is
    # piecewise trilinear, so the step costs no accuracy otherwise)
    h = 1e-4
    fd = np.zeros_like(f)
    for idx in np.ndindex(f.shape):
        e = np.zeros_like(f)
        e[idx] = h
        fd[idx] = (objective(f + e) - objective(f - e)) / (2 * h)
    np.testing.assert_allclose(g, fd, atol=3e-3 * np.abs(fd).max())


def test_pose_gradient_with_field_matches_finite_differences():
    """d/d(bend, twist, taper) at fixed deformed points when a field sits
    under the pose, against central differences of the chain."""
    net = S.NetConfig(levels=2, log2_table=6, pe_bands=1, base_res=2)
    rng = np.random.default_rng(13)
    tables = rng.uniform(-1, 1, (net.levels, 1 << net.log2_table, net.feats))
    f = _random_field(4, 14, lip=0.35)
    pose = np.array([0.4, -0.6, 0.3])
    p0 = rng.uniform(0.1, 0.9, (20, 3))
    p1 = np.clip(p0 + rng.normal(0, 0.05, (20, 3)), 0.05, 0.95)
    x0, x1 = O.deform_field(pose, f, p0), O.deform_field(pose, f, p1)
    df = rng.normal(size=(20, net.in_dim))

    def objective(th):
        q0, q1 = O.inverse_field(th, f, x0), O.inverse_field(th, f, x1)
        return float((df * O.encode_segments(net, tables, q0, q1)).sum())

    g = O.pose_gradient(net, tables, pose, O.inverse_field(pose, f, x0), O.inverse_field(pose, f, x1), df, field=f)
    h = 1e-3                         # the oracle's FP32 cell coordinate quantises the forward at ~1e-7
    fd = np.array([(objective(pose + h * e) - objective(pose - h * e)) / (2 * h) for e in np.eye(3)])
    np.testing.assert_allclose(g, fd, atol=3e-3 * np.abs(fd).max())
