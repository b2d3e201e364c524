"""Pins of the oracle's geometry (Sec. III-A: SDF definition, generation by sampling a
mesh, trilinear lookup) against closed forms, brute force and bounds that do not come
from the oracle itself."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


# ---------------------------------------------------------------- closest point on a triangle
def _brute_distance(p, a, b, c, n=400):
    """Distance to a dense barycentric sampling of the triangle (an upper bound that
    converges to the exact distance as n grows)."""
    u, v = np.meshgrid(np.linspace(0, 1, n + 1), np.linspace(0, 1, n + 1))
    m = (u + v) <= 1.0
    u, v = u[m], v[m]
    pts = a[None] + u[:, None] * (b - a)[None] + v[:, None] * (c - a)[None]
    return np.min(np.linalg.norm(pts - p[None], axis=1))


def test_closest_point_matches_brute_force():
    rng = np.random.default_rng(1)
    for _ in range(60):
        a, b, c = rng.normal(size=(3, 3))
        p = rng.normal(size=3) * 2
        q, region = O.closest_point_triangle(p, a, b, c)
        d = np.linalg.norm(p - q)
        brute = _brute_distance(p, a, b, c)
        # sampling bound: half the longest sample spacing
        h = max(np.linalg.norm(b - a), np.linalg.norm(c - a), np.linalg.norm(c - b)) / 400
        assert d <= brute + 1e-12
        assert brute <= d + h
        # q lies in the triangle: barycentric coordinates in [0, 1]
        M = np.stack([b - a, c - a], 1)
        st, *_ = np.linalg.lstsq(M, q - a, rcond=None)
        assert st.min() >= -1e-9 and st.sum() <= 1 + 1e-9


def test_closest_point_regions_by_construction():
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    cases = [((0.2, 0.2, 1.0), 0, (0.2, 0.2, 0)), ((-1, -1, 0.5), 1, (0, 0, 0)),
             ((2, -0.5, 0), 2, (1, 0, 0)), ((-0.2, 3, 0), 3, (0, 1, 0)),
             ((0.5, -1, 0.3), 4, (0.5, 0, 0)), ((1, 1, 0), 5, (0.5, 0.5, 0)),
             ((-1, 0.25, 0), 6, (0, 0.25, 0))]
    for p, reg, q_exp in cases:
        q, r = O.closest_point_triangle(p, a, b, c)
        assert r == reg, (p, r)
        np.testing.assert_allclose(q, q_exp, atol=1e-15)


# ---------------------------------------------------------------- solid angle, winding number
def test_solid_angle_octant():
    # the triangle (e_x, e_y, e_z) seen from the origin covers one eighth of the sphere
    assert O.solid_angle([0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]) == pytest.approx(math.pi / 2, abs=1e-14)
    assert O.solid_angle([0, 0, 0], [1, 0, 0], [0, 0, 1], [0, 1, 0]) == pytest.approx(-math.pi / 2, abs=1e-14)


@pytest.mark.parametrize("mesh", ["box", "ico", "hole"])
def test_winding_number_inside_outside(mesh):
    if mesh == "box":
        V, T = S.box_mesh(0.01, 0.02, 0.03)
        inside, outside = [(0.001, -0.01, 0.02)], [(0.02, 0, 0), (0, 0, -0.05)]
    elif mesh == "ico":
        V, T = S.icosphere(0.01, 2)
        inside, outside = [(0.002, 0.003, -0.001)], [(0.011, 0, 0), (0.02, 0.02, 0.0)]
    else:
        V, T = S.box_with_hole_mesh(24e-3, 24e-3, 16e-3, 4.1e-3, 12e-3, 168)
        inside, outside = [(8e-3, 8e-3, -8e-3), (0, 0, -14e-3)], [(0, 0, -6e-3), (0, 0, 1e-3)]
    for p in inside:
        assert O.winding_number(p, V, T) == pytest.approx(1.0, abs=1e-12)
    for p in outside:
        assert O.winding_number(p, V, T) == pytest.approx(0.0, abs=1e-12)


# ---------------------------------------------------------------- baked SDFs vs analytic SDFs
def _box_sdf(x, b):
    q = np.abs(x) - b
    outside = np.linalg.norm(np.maximum(q, 0), axis=-1)
    inside = np.minimum(np.max(q, axis=-1), 0)
    return outside + inside


def _node_positions(lo, h, dims):
    i = np.arange(dims[0]) * np.float64(h) + np.float64(lo[0])
    j = np.arange(dims[1]) * np.float64(h) + np.float64(lo[1])
    k = np.arange(dims[2]) * np.float64(h) + np.float64(lo[2])
    Z, Y, X = np.meshgrid(k, j, i, indexing="ij")
    return np.stack([X, Y, Z], -1)


def test_box_bake_equals_analytic_box_sdf():
    V, T = S.box_mesh(0.01, 0.015, 0.02)
    b = V.max(0).astype(np.float64)   # the float32 corners are the exact box
    lo, h, dims = O.grid_params(V, 20, 3e-3)
    phi = O.bake_nodes(V, T, lo, h, dims)
    X = _node_positions(lo, h, dims)
    np.testing.assert_allclose(phi, _box_sdf(X, b), rtol=0, atol=1e-15)


def test_sphere_bake_within_faceting_bound():
    r = 0.01
    V, T = S.icosphere(r, 2)
    Vd = V.astype(np.float64)
    a, bb, c = Vd[T[:, 0]], Vd[T[:, 1]], Vd[T[:, 2]]
    nrm = np.cross(bb - a, c - a)
    r_in = np.min(np.abs(np.einsum("ij,ij->i", nrm / np.linalg.norm(nrm, axis=1)[:, None], a)))
    r_out = np.max(np.linalg.norm(Vd, axis=1))
    lo, h, dims = O.grid_params(V, 16, 2e-3)
    phi = O.bake_nodes(V, T, lo, h, dims)
    R = np.linalg.norm(_node_positions(lo, h, dims), axis=-1)
    # the mesh solid lies between the balls of radius r_in and r_out, so its signed
    # distance lies between theirs
    assert np.all(phi >= R - r_out - 1e-12)
    assert np.all(phi <= R - r_in + 1e-12)
    assert r_out - r_in < 0.05 * r


def _capped_cylinder_sdf(x, r, hh):
    d = np.stack([np.linalg.norm(x[..., :2], axis=-1) - r, np.abs(x[..., 2]) - hh], -1)
    return np.minimum(np.max(d, -1), 0) + np.linalg.norm(np.maximum(d, 0), axis=-1)


def test_cylinder_bake_between_inscribed_and_circumscribed():
    r, hgt, n = 4e-3, 25e-3, 32
    V, T = S.cylinder_mesh(r, hgt, n)
    lo, h, dims = O.grid_params(V, 14, 1e-3)
    phi = O.bake_nodes(V, T, lo, h, dims)
    X = _node_positions(lo, h, dims)
    # bounds from the float32 vertices: circumscribed radius, and the inscribed radius as
    # the smallest distance from the axis to a side's line
    bottom = V[(V[:, 2] == V[:, 2].min()) & (np.linalg.norm(V[:, :2], axis=1) > 0)]
    ring = bottom[:, :2].astype(np.float64)
    assert len(ring) == n
    ang = np.arctan2(ring[:, 1], ring[:, 0])
    ring = ring[np.argsort(ang)]
    a, b = ring, np.roll(ring, -1, 0)
    r_in = np.min(np.abs(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]) / np.linalg.norm(b - a, axis=1))
    r_out = np.max(np.linalg.norm(ring, axis=1))
    hh = float(V[:, 2].max())
    outer = _capped_cylinder_sdf(X, r_out, hh)
    inner = _capped_cylinder_sdf(X, r_in, hh)
    assert r_in == pytest.approx(r * math.cos(math.pi / n), rel=1e-6)
    assert np.all(phi >= outer - 1e-12)
    assert np.all(phi <= inner + 1e-12)


def test_sampled_nodes_equal_full_bake():
    V, T = S.box_with_hole_mesh(24e-3, 24e-3, 16e-3, 4.1e-3, 12e-3, 168)
    lo, h, dims = O.grid_params(V, 12, 1e-3)
    full = O.bake_nodes(V, T, lo, h, dims).reshape(-1)
    nodes = np.random.default_rng(0).choice(full.size, 50, replace=False)
    np.testing.assert_array_equal(O.bake_nodes(V, T, lo, h, dims, nodes), full[nodes])


def test_grid_params_cover_padded_box():
    V, T = S.bolt_mesh()
    for res, pad in ((64, 1e-3), (256, 1e-3), (33, 2e-3)):
        lo, h, dims = O.grid_params(V, res, pad)
        assert tuple(dims) == (res, res, res)
        hi = lo.astype(np.float64) + (res - 1) * np.float64(h)
        mn, mx = V.min(0).astype(np.float64), V.max(0).astype(np.float64)
        # every axis covers the padded box (to float32 rounding of lo and h)
        assert np.all(lo <= mn - pad + 1e-6) and np.all(hi >= mx + pad - 1e-6)
        # the longest axis is spanned exactly: h = L / (res - 1)
        L = np.max(mx - mn + 2 * pad)
        assert abs(np.float64(h) * (res - 1) - L) <= 1e-6 * L


# ---------------------------------------------------------------- trilinear lookup
def test_trilinear_reproduces_affine_field_exactly():
    rng = np.random.default_rng(2)
    dims = np.array([7, 5, 9], np.int32)
    lo = np.array([-0.01, 0.02, -0.03], np.float32)
    h = np.float32(0.0025)
    n = rng.normal(size=3)
    c0 = 0.004
    X = _node_positions(lo, h, dims)
    grid = X @ n - c0
    pts = (lo + rng.uniform(0, 1, (500, 3)) * (dims - 1) * h).astype(np.float32)
    phi, grad, valid = O.query(grid, lo, h, dims, pts)
    assert valid.all()
    np.testing.assert_allclose(phi, pts.astype(np.float64) @ n - c0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(grad, np.broadcast_to(n, grad.shape), rtol=0, atol=1e-12)


def test_trilinear_at_nodes_and_outside():
    rng = np.random.default_rng(3)
    dims = np.array([4, 6, 5], np.int32)
    lo = np.zeros(3, np.float32)
    h = np.float32(0.5)
    grid = rng.normal(size=(dims[2], dims[1], dims[0]))
    ijk = np.stack([rng.integers(0, d, 40) for d in dims], 1)
    pts = (ijk * 0.5).astype(np.float32)
    phi, _, valid = O.query(grid, lo, h, dims, pts)
    assert valid.all()
    np.testing.assert_array_equal(phi, grid[ijk[:, 2], ijk[:, 1], ijk[:, 0]])
    out = np.array([[-1e-3, 1, 1], [1, 1, 2.0001], [1.5, 2.5 + 0.01, 1]], np.float32)
    _, _, valid = O.query(grid, lo, h, dims, out)
    assert not valid.any()


def test_trilinear_gradient_is_derivative_of_value():
    """Inside a cell the interpolant is smooth, so a central difference of the returned
    value must match the returned gradient."""
    rng = np.random.default_rng(4)
    dims = np.array([5, 5, 5], np.int32)
    lo = np.zeros(3, np.float32)
    h = np.float32(1.0)
    grid = rng.normal(size=(5, 5, 5))
    for _ in range(30):
        cell = rng.integers(0, 4, 3)
        x = cell + rng.uniform(0.2, 0.8, 3)
        _, g, _ = O.query(grid, lo, h, dims, x[None].astype(np.float32))
        # use float64 evaluation through points that are exact in float32
        eps = 2.0 ** -12
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a] += eps
            xm[a] -= eps
            fp, _, _ = O.query(grid, lo, h, dims, xp[None].astype(np.float32))
            fm, _, _ = O.query(grid, lo, h, dims, xm[None].astype(np.float32))
            dxa = np.float64(np.float32(xp[a])) - np.float64(np.float32(xm[a]))
            assert (fp[0] - fm[0]) / dxa == pytest.approx(g[0, a], abs=1e-9)


# ---------------------------------------------------------------- mass properties
def test_mass_properties_box_closed_form():
    hx, hy, hz = 0.01, 0.02, 0.03
    V, T = S.box_mesh(hx, hy, hz)
    m, com, I = O.mass_properties(V, T, 1000.0)
    a, b, c = 2 * hx, 2 * hy, 2 * hz
    M = 1000.0 * a * b * c
    assert m == pytest.approx(M, rel=1e-6)
    np.testing.assert_allclose(com, 0, atol=1e-12)
    np.testing.assert_allclose(I, np.diag([M / 12 * (b * b + c * c), M / 12 * (a * a + c * c),
                                           M / 12 * (a * a + b * b)]), rtol=1e-6, atol=1e-15)


def test_mass_properties_offset_box_parallel_axis():
    V, T = S.box_mesh(0.01, 0.01, 0.01)
    V2 = (V.astype(np.float64) + [0.05, -0.02, 0.01]).astype(np.float32)
    m1, c1, I1 = O.mass_properties(V, T, 500.0)
    m2, c2, I2 = O.mass_properties(V2, T, 500.0)
    # the float32 translation changes the box edges by float32 rounding only
    assert m2 == pytest.approx(m1, rel=1e-6)
    np.testing.assert_allclose(c2, [0.05, -0.02, 0.01], atol=1e-8)
    np.testing.assert_allclose(I2, I1, rtol=1e-5, atol=1e-14)


def test_mass_properties_regular_prism_closed_form():
    r, hgt, n, rho = 4e-3, 25e-3, 16, 7800.0
    V, T = S.cylinder_mesh(r, hgt, n)
    m, com, I = O.mass_properties(V, T, rho)
    area = 0.5 * n * r * r * math.sin(2 * math.pi / n)
    # polar second moment of a regular n-gon of circumradius r about its centre
    J = n * r ** 4 / 12 * math.sin(2 * math.pi / n) * (2 + math.cos(2 * math.pi / n))
    M = rho * area * hgt
    assert m == pytest.approx(M, rel=1e-6)
    np.testing.assert_allclose(com, 0, atol=1e-10)
    assert I[2, 2] == pytest.approx(rho * hgt * J, rel=1e-5)
    assert I[0, 0] == pytest.approx(rho * hgt * J / 2 + M * hgt * hgt / 12, rel=1e-5)
    assert I[1, 1] == pytest.approx(I[0, 0], rel=1e-5)


def test_torus_mass_properties_converge_to_closed_form():
    """The pile torus (R = 15.4 mm, r = 8 mm): a closed, outward-wound surface whose
    polyhedral volume and axial / transverse moments approach the solid torus's closed
    forms, V = 2 pi^2 R r^2, I_zz = m (R^2 + 3 r^2 / 4), I_xx = m (R^2 / 2 + 5 r^2 / 8), as the
    segmentation is refined (error of order the squared segment angle)."""
    R, r = 15.4e-3, 8.0e-3
    errs = []
    for n_u, n_v in ((64, 16), (256, 64)):
        V, T = S.torus_mesh(R, r, n_u, n_v)
        assert S.edge_manifold_check(T) and S.signed_volume(V, T) > 0
        m, com, I = O.mass_properties(V, T, 1.0)
        vol = 2 * math.pi ** 2 * R * r * r
        np.testing.assert_allclose(com, 0, atol=1e-9)
        e = [abs(m / vol - 1), abs(I[2, 2] / (m * (R * R + 0.75 * r * r)) - 1),
             abs(I[0, 0] / (m * (0.5 * R * R + 0.625 * r * r)) - 1)]
        errs.append(max(e))
    assert errs[0] < 0.04 and errs[1] < 0.003 and errs[1] < errs[0] / 8, errs


def test_bowl_mass_properties_converge_to_closed_form():
    """The pile bowl (rim 50 mm, depth 29 mm, wall 2 mm): a closed, outward-wound shell
    between two concentric spherical caps whose volume approaches the difference of the
    caps' closed forms pi h^2 (3 R - h) / 3 as the rings and segments are refined, with its
    centre of mass on the axis."""
    rim, depth, wall = 50e-3, 29e-3, 2e-3
    Ro = (rim * rim + depth * depth) / (2 * depth)
    Ri = Ro - wall
    cap = lambda Rs, h: math.pi * h * h * (3 * Rs - h) / 3
    vol = cap(Ro, depth) - cap(Ri, depth - wall)
    errs = []
    for n_seg, n_ring in ((32, 9), (128, 36)):
        V, T = S.bowl_mesh(rim, depth, wall, n_seg, n_ring)
        assert S.edge_manifold_check(T) and S.signed_volume(V, T) > 0
        m, com, I = O.mass_properties(V, T, 1.0)
        np.testing.assert_allclose(com[:2], 0, atol=1e-9)
        assert 0 < com[2] < depth
        errs.append(abs(m / vol - 1))
    assert errs[0] < 0.03 and errs[1] < 0.003 and errs[1] < errs[0] / 8, errs
