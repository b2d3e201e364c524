"""Per-triangle contact generation on the GPU (contact_gen = 1: one candidate per face of
the point body's mesh, the minimiser of the opposing SDF over the face by projected
gradient descent with adaptive steps, Sec. III-A) against the FP64 oracle.

Tolerances.  With the same step decisions the two sides differ by the rounding of the pose
transform and the lookups, as in the sample narrow phase (5e-5 h in phi), plus the
float32 rounding of the descent's steps; a late accept/reject decision that falls the
other way (most of a face's last decisions are near-ties: the step has shrunk to a tiny
fraction of a voxel) moves the minimiser by at most that step.  So per face: validity
equal; phi within 1e-4 h for 99% of the faces and within 2e-3 h for all (a decision that
flips at a larger step moves phi by that step times the in-plane slope); x within 1e-6 m
for 99% of the faces, and beyond 1e-5 m for at most 1% -- on a face lying along a flat
stretch of the SDF every point of the stretch is a minimiser, and one flipped early
decision ends elsewhere on it with the same phi.  Contact sets of a whole pair then agree
in bulk.  Near-tie face decisions are the rule here, not the exception, so after one
frame of the peg the contact sets may differ by a face or two: positions stay within
2e-4 m, orientations within 2e-3 rad for 75% of the envs and 1e-2 rad for all.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


def _fw():
    from paper_2205_03532_b300 import fw
    return fw


def _peg_scene(n_envs=8, seed=7):
    sc = S.peg_in_hole_scene(n_envs=n_envs, seed=seed)
    b = sc.groups[0].bodies
    rng = np.random.default_rng(seed)
    b["pos"][:, 0, 2] = 12.5e-3 + rng.uniform(-4e-3, 0.3e-3, len(b))
    b["pos"][:, 0, :2] = rng.uniform(-0.09e-3, 0.09e-3, (len(b), 2))
    for e in range(len(b)):
        tilt = np.deg2rad(rng.uniform(-0.3, 0.3, 2))
        b["quat"][e, 0] = S.quat_mul(S.quat_axis_angle([1, 0, 0], tilt[0]), S.quat_axis_angle([0, 1, 0], tilt[1]))
    return sc


@pytest.fixture(scope="module")
def tri_pair():
    fw = _fw()
    sc = _peg_scene()
    gw = fw.world_from_scene(sc, contact_gen=1, tri_iters=16)
    ow = O.world_from_scene(sc, contact_gen=1, tri_iters=16)
    return sc, gw, ow


def test_each_face_matches_the_oracle(tri_pair):
    sc, gw, ow = tri_pair
    h = float(gw.get_sdf(1, values=False)[1])
    nt = len(sc.assets[0].tris)
    dx_all, dphi_all = [], []
    for env in range(sc.n_envs):
        gx, gphi, gn = gw.tri_contacts(env, 0, nt)
        ox, ophi, on, ov, _ = ow.tri_contacts(env, 0, nt)
        gv = np.isfinite(gphi)
        assert np.array_equal(gv, ov), env
        dphi = np.abs(gphi[gv] - ophi[gv])
        assert np.all(dphi <= 2e-3 * h), (env, float(dphi.max() / h))
        dphi_all.append(dphi)
        dx_all.append(np.linalg.norm(gx[gv] - ox[gv], axis=1))
        assert np.all(np.abs(np.linalg.norm(gn[gv], axis=1) - 1) <= 1e-5)
    dx_all, dphi_all = np.concatenate(dx_all), np.concatenate(dphi_all)
    assert np.percentile(dx_all, 99) <= 1e-6, float(np.percentile(dx_all, 99))
    assert np.mean(dx_all > 1e-5) <= 0.01, float(np.mean(dx_all > 1e-5))
    assert np.percentile(dphi_all, 99) <= 1e-4 * h, float(np.percentile(dphi_all, 99) / h)


def test_affine_field_ends_on_the_lowest_vertex():
    """phi = m.x - c on the grid: each face's minimum is its lowest vertex (the descent
    reaches it through the face projection), on the GPU as in the oracle."""
    fw = _fw()
    m = np.array([0.3, -0.5, 0.81])
    m /= np.linalg.norm(m)
    n, h = 48, np.float32(4e-4)
    lo = np.full(3, -0.5 * (n - 1) * h, np.float32)
    i = lo[0] + np.arange(n) * np.float64(h)
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    vals = (m[0] * X + m[1] * Y + m[2] * Z - 1e-3).astype(np.float32)
    V = 4e-3 * np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 1.0, 0.05], [0.3, 0.25, 1.0]], np.float32)
    T = np.array([[0, 2, 1], [0, 1, 3], [1, 2, 3], [0, 3, 2]], np.int32)
    w = fw.World(contact_gen=1, tri_iters=24)
    a = w.add_mesh_asset(V, T, None)
    GV, GT = S.box_mesh(0.02, 0.02, 0.02)
    bsdf = w.add_mesh_asset(GV, GT, None)
    w.set_sdf(bsdf, lo, h, np.array([n, n, n], np.int32), vals)
    q = S.quat_axis_angle([0.2, 1.0, -0.4], 0.7)
    bodies = np.zeros((1, 2), S.BODY_DTYPE)
    bodies[0, 0] = S._body(a, S.STATIC, (-1.5e-3, 1e-3, -2e-3), q, 0.5)
    bodies[0, 1] = S._body(bsdf, S.STATIC, (0, 0, 0), (0, 0, 0, 1), 0.5)
    w.add_env_bodies(bodies, np.array([[0, 1]], np.int32))
    x, phi, nrm = w.tri_contacts(0, 0, len(T))
    qd = bodies[0, 0]["quat"].astype(np.float64)
    qx, qy, qz, qw = qd / np.linalg.norm(qd)
    R = np.array([[1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
                  [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
                  [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)]])
    Vw = V.astype(np.float64) @ R.T + bodies[0, 0]["pos"].astype(np.float64)
    for t in range(len(T)):
        F = Vw[T[t]]
        k = int(np.argmin(F @ m))
        assert np.linalg.norm(x[t] - F[k]) <= 1e-7, (t, x[t], F[k])
        assert abs(phi[t] - (F[k] @ m - 1e-3)) <= 1e-7
        np.testing.assert_allclose(nrm[t], m, atol=1e-5)


def test_collide_agrees_with_the_oracle(tri_pair):
    sc, gw, ow = tri_pair
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    gw.collide()
    ow.collide()
    identical = 0
    for env in range(sc.n_envs):
        gc = gw.get_contacts(env)
        oc, _, _ = ow.contacts(env)
        assert len(oc) > 0
        common = len(set(gc["sample"]) & set(oc["sample"]))
        assert common >= 0.9 * max(len(gc), len(oc)), (env, common, len(gc), len(oc))
        assert abs(len(gc) - len(oc)) <= max(2, 0.1 * len(oc))
        identical += int(list(gc["sample"]) == list(oc["sample"]) and list(gc["patch"]) == list(oc["patch"]))
    assert identical >= sc.n_envs // 2, identical


def _rot_angle(q1, q2):
    d = abs(float(np.dot(q1 / np.linalg.norm(q1), q2 / np.linalg.norm(q2))))
    return 2 * math.acos(min(1.0, d))


def test_one_frame_with_per_triangle_contacts():
    fw = _fw()
    sc = _peg_scene(n_envs=16, seed=3)
    gw = fw.world_from_scene(sc, contact_gen=1, tri_iters=16)
    ow = O.world_from_scene(sc, contact_gen=1, tri_iters=16)
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    gw.step(sc.sim.n_substeps, sc.sim.n_iters)
    ow.step(sc.sim.n_substeps, sc.sim.n_iters)
    gp, gq = gw.get_state()[:2]
    op, oq = ow.state()[:2]
    rot = []
    for i in range(0, len(gp), 2):
        assert np.linalg.norm(gp[i] - op[i]) <= 2e-4, (i, gp[i], op[i])
        rot.append(_rot_angle(gq[i].astype(np.float64), oq[i]))
    rot = np.array(rot)
    assert np.all(rot <= 1e-2) and np.mean(rot <= 2e-3) >= 0.75, rot
    gw.close()


def test_substep_generate_equals_the_per_face_hook(tri_pair):
    """The substep's Generate (each thread streams the descent steps of its four faces)
    and the per-face hook (one face per thread) take the same steps: every contact's
    point and phi equal the hook's for its face bit for bit; the normal, the same
    expression compiled in two places, to a couple of float32 ulps."""
    sc, gw, ow = tri_pair
    nt = len(sc.assets[0].tris)
    gw.collide()
    checked = 0
    for env in range(sc.n_envs):
        c = gw.get_contacts(env)
        x, phi, nrm = gw.tri_contacts(env, 0, nt)
        f = c["sample"]
        np.testing.assert_array_equal(c["xa"], x[f])
        np.testing.assert_array_equal(c["phi"], phi[f])
        np.testing.assert_allclose(c["n"], nrm[f], rtol=0, atol=2.5e-7)
        checked += len(c)
    assert checked > 50
