"""Velocity iterations (n_vel_iters: bias-free sweeps after the integration, the paper's
"velocity iterations" of its position / velocity iteration counts) in the oracle, pinned
by what they must and must not change rather than by the oracle's own code:

  * they run after the positions are integrated, so positions and orientations are
    exactly those of the same substep without them;
  * a box resting slightly sunk into the ground leaves the position sweeps with the
    separating velocity the bias asked for; bias-free sweeps take it back (the accumulated
    normal impulse can shrink), leaving the box nearly at rest;
  * frictionless free bodies keep their total linear momentum, and their angular
    momentum taken about the substep's starting centres of mass (the velocity sweeps act
    with the rows' lever arms from the substep's start).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


def _box_on_ground(n_vel, sink=2e-4, mu=0.5, gravity=(0, 0, -9.81)):
    V, T = S.box_mesh(0.01, 0.01, 0.01)
    Sp = S.sample_surface(V, T, 600, np.random.default_rng(0))
    GV, GT = S.box_mesh(0.2, 0.2, 0.01)
    w = O.OracleWorld(gravity=gravity, n_vel_iters=n_vel)
    a = w.add_asset(V, T, Sp)
    g = w.add_asset(GV, GT, None)
    w.bake(g, 96, 2e-3)
    b = np.zeros((1, 2), S.BODY_DTYPE)
    b[0, 0] = S._body(a, S.DYNAMIC, (0, 0, 0.01 - sink), (0, 0, 0, 1), mu)
    b[0, 1] = S._body(g, S.STATIC, (0, 0, -0.01), (0, 0, 0, 1), mu)
    w.add_envs(b, np.array([[0, 1]], np.int32))
    return w


def test_positions_are_those_without_velocity_iterations():
    s0, s1 = [], []
    for n_vel, out in ((0, s0), (4, s1)):
        w = _box_on_ground(n_vel)
        w.substep(1 / 480, 16)
        out.extend(w.state())
    np.testing.assert_array_equal(s1[0], s0[0])
    np.testing.assert_array_equal(s1[1], s0[1])
    assert np.abs(s1[2] - s0[2]).max() > 1e-4      # the velocities did change


def test_velocity_iterations_remove_the_bias_velocity():
    vz = {}
    for n_vel in (0, 16):
        w = _box_on_ground(n_vel)
        w.substep(1 / 480, 16)
        vz[n_vel] = w.state()[2][0, 2]
    assert vz[0] > 0.015                             # pushed out by the bias, 0.2 x 0.2 mm x 480 /s
    assert abs(vz[16]) <= 0.05 * vz[0], vz


@pytest.mark.parametrize("solver", [0, 1])
def test_frictionless_momentum_with_velocity_iterations(solver):
    V, T = S.box_mesh(0.01, 0.01, 0.01)
    Sp = S.sample_surface(V, T, 300, np.random.default_rng(1))
    w = O.OracleWorld(gravity=(0, 0, 0), n_vel_iters=3, solver=solver)
    a = w.add_asset(V, T, Sp)
    b = w.add_asset(V, T, Sp)
    bodies = np.zeros((1, 2), S.BODY_DTYPE)
    bodies[0, 0] = S._body(a, S.DYNAMIC, (0, 0, 0), (0, 0, 0, 1), 0.0, 0.0, (0.3, 0.05, 0), (0.2, -0.1, 0.4))
    bodies[0, 1] = S._body(b, S.DYNAMIC, (0.02, 0.001, 0.002), (0, 0, 0, 1), 0.0, 0.0, (-0.2, 0, 0.01), (0, 0.3, 0))
    w.add_envs(bodies, np.array([[0, 1]], np.int32))
    xa = np.array([[0.01, 0.002, 0.004], [0.01, -0.006, -0.001], [0.0095, 0.004, -0.008]])
    nrm = np.array([[-1.0, 0.05, 0.0], [-1.0, 0.0, 0.1], [-0.98, -0.1, 0.05]])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    c = np.zeros(3, O.CONTACT_DTYPE)
    c["sample"], c["xa"], c["n"], c["phi"] = np.arange(3), xa, nrm, [-1e-5, -3e-5, 2e-6]
    c["xb"] = c["xa"] - c["phi"][:, None] * c["n"]
    p0, q0, v0, w0 = w.state()
    w.set_contacts(0, c)
    w.substep(1 / 240, 6, detect=False)
    p1, q1, v1, w1 = w.state()
    m = w.mass(0)[0]
    I = w.mass(0)[2][0, 0]
    assert np.abs(v1 - v0).max() > 1e-4
    np.testing.assert_allclose(m * v1.sum(0), m * v0.sum(0), rtol=0, atol=1e-15)
    L0 = (I * w0 + m * np.cross(p0, v0)).sum(0)
    L1 = (I * w1 + m * np.cross(p0, v1)).sum(0)    # about the starting centres (cubes: com = pos)
    np.testing.assert_allclose(L1, L0, rtol=0, atol=1e-16)
