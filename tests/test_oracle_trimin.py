"""The oracle's per-triangle contact generator (one contact per face of the point body's
mesh by local minimisation over the face, Sec. III-A), pinned without the oracle's own
code:

  * an affine field phi = m.x - c (trilinear interpolation reproduces it exactly): the
    minimum of an affine function over a triangle is at its lowest vertex, so every face's
    result is that vertex (to 1e-12 m), with phi = m.v - c;
  * a baked sphere distance: on every face the descent finds a value at least as low as
    brute force over a dense barycentric grid of the face (evaluated with the plain
    trilinear query), within a small fraction of a voxel;
  * through collide: every contact lies on its own face, and its normal is the unit SDF
    gradient there.
"""
import numpy as np

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


def _tet(scale=4e-3):
    V = scale * np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 1.0, 0.05], [0.3, 0.25, 1.0]], np.float32)
    # outward winding
    T = np.array([[0, 2, 1], [0, 1, 3], [1, 2, 3], [0, 3, 2]], np.int32)
    c = V.mean(axis=0)
    for t in range(4):
        a, b, d = V[T[t]]
        if np.dot(np.cross(b - a, d - a), a - c) < 0:
            T[t] = T[t][[0, 2, 1]]
    return V, T


def _world_with_grid(V, T, lo, h, dims, vals, q_a, p_a):
    w = O.OracleWorld(contact_gen=1, tri_iters=24)
    a = w.add_asset(V, T, None)
    GV, GT = S.box_mesh(0.02, 0.02, 0.02)
    b = w.add_asset(GV, GT, None)
    w.set_grid(b, lo, h, dims, vals)
    bodies = np.zeros((1, 2), S.BODY_DTYPE)
    bodies[0, 0] = S._body(a, S.STATIC, p_a, q_a, 0.5)
    bodies[0, 1] = S._body(b, S.STATIC, (0.0, 0.0, 0.0), (0, 0, 0, 1), 0.5)
    w.add_envs(bodies, np.array([[0, 1]], np.int32))
    return w


def _grid(f, n=48, h=4e-4):
    lo = np.full(3, -0.5 * (n - 1) * h, np.float32)
    dims = np.array([n, n, n], np.int32)
    i = lo[0] + np.arange(n) * np.float64(h)
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    return lo, np.float32(h), dims, f(X, Y, Z).astype(np.float32)


def _faces_world(V, T, q, p):
    """the faces in the world frame (body b sits at the identity); q, p as the world
    stores them (float32), the rotation of the unit quaternion in float64"""
    q = np.asarray(q, np.float32).astype(np.float64)
    x, y, z, w_ = q / np.linalg.norm(q)
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w_), 2 * (x * z + y * w_)],
                  [2 * (x * y + z * w_), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w_)],
                  [2 * (x * z - y * w_), 2 * (y * z + x * w_), 1 - 2 * (x * x + y * y)]])
    Vw = V.astype(np.float64) @ R.T + np.asarray(p, np.float32).astype(np.float64)
    return Vw[T]


def test_affine_field_minimum_is_the_lowest_vertex():
    m = np.array([0.3, -0.5, 0.81])
    m /= np.linalg.norm(m)
    lo, h, dims, vals = _grid(lambda X, Y, Z: m[0] * X + m[1] * Y + m[2] * Z - 1e-3)
    V, T = _tet()
    q = S.quat_axis_angle([0.2, 1.0, -0.4], 0.7)
    p = (-1.5e-3, 1e-3, -2e-3)
    w = _world_with_grid(V, T, lo, h, dims, vals, q, p)
    x, phi, n, valid, margin = w.tri_contacts(0, 0, len(T))
    F = _faces_world(V, T, q, p)
    assert valid.all()
    for t in range(len(T)):
        heights = F[t] @ m
        k = int(np.argmin(heights))
        # the vertex itself (the descent ends on it through the face projection)
        np.testing.assert_allclose(x[t], F[t][k], rtol=0, atol=1e-12)
        # phi: the affine field at that vertex (trilinear is exact on an affine field,
        # up to the float32 rounding of the stored node values)
        assert abs(phi[t] - (heights[k] - 1e-3)) <= 1e-7, (t, phi[t], heights[k] - 1e-3)
        np.testing.assert_allclose(n[t], m, atol=1e-5)


def test_sphere_field_descent_beats_dense_sampling():
    r0 = 3e-3
    lo, h, dims, vals = _grid(lambda X, Y, Z: np.sqrt(X * X + Y * Y + Z * Z) - r0)
    V, T = _tet(scale=3e-3)
    q = S.quat_axis_angle([1.0, 0.3, 0.2], 0.4)
    p = (-2e-3, -1.5e-3, 1.2e-3)
    w = _world_with_grid(V, T, lo, h, dims, vals, q, p)
    x, phi, n, valid, margin = w.tri_contacts(0, 0, len(T))
    F = _faces_world(V, T, q, p)
    k = 60
    uu, vv = np.meshgrid(np.arange(k + 1), np.arange(k + 1), indexing="ij")
    keep = uu + vv <= k
    bar = np.stack([1 - (uu[keep] + vv[keep]) / k, uu[keep] / k, vv[keep] / k], axis=1)
    for t in range(len(T)):
        pts = (bar @ F[t]).astype(np.float32)
        bphi, _, bvalid = O.query(vals.astype(np.float64), lo, h, dims, pts)
        best = bphi[bvalid].min()
        assert valid[t]
        assert phi[t] <= best + 0.01 * h, (t, phi[t], best)
        # the result is a point of the face with that value
        rphi, _, _ = O.query(vals.astype(np.float64), lo, h, dims, x[t:t + 1].astype(np.float32))
        assert abs(rphi[0] - phi[t]) <= 1e-6 * h + 1e-9


def test_collide_contacts_lie_on_their_faces():
    sc = S.peg_in_hole_scene(n_envs=2, seed=4)
    b = sc.groups[0].bodies
    b["pos"][:, 0, 2] = 12.5e-3 - 2e-3
    w = O.world_from_scene(sc, contact_gen=1, tri_iters=16)
    w.collide()
    peg = sc.assets[0]
    Vp, Tp = peg.verts.astype(np.float64), peg.tris
    for env in range(2):
        c, _, _ = w.contacts(env)
        assert len(c) > 0 and np.all(c["sample"] < len(Tp))
        q, p = b["quat"][env, 0], b["pos"][env, 0]
        F = _faces_world(Vp, Tp, q, p)
        for row in c:
            a, bb, cc = F[row["sample"]]
            nrm = np.cross(bb - a, cc - a)
            nrm /= np.linalg.norm(nrm)
            assert abs(np.dot(row["xa"] - a, nrm)) <= 1e-9          # in the face's plane
            # barycentric coordinates within [0, 1]
            M = np.stack([bb - a, cc - a], axis=1)
            uv = np.linalg.lstsq(M, row["xa"] - a, rcond=None)[0]
            assert uv.min() >= -1e-9 and uv.sum() <= 1 + 1e-9, uv
            np.testing.assert_allclose(np.linalg.norm(row["n"]), 1.0, atol=1e-12)
