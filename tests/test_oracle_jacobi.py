"""The oracle's Jacobi solver (every contact's block update from the sweep-start
velocities, all taken with the weight 1 / active contacts), pinned against the
Gauss-Seidel solver and physical invariants rather than its own code:

  * one contact: the weight is 1 and a Jacobi sweep is a Gauss-Seidel sweep;
  * frictionless two free bodies: equal and opposite impulses conserve linear and angular
    momentum whatever the number of sweeps;
  * a resting box: with enough sweeps Jacobi reaches the velocities Gauss-Seidel converges
    to (the constrained velocity components are unique);
  * Coulomb: every row's impulse stays in the friction cone.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


def _cube(half=0.01, n=600, seed=0):
    V, T = S.box_mesh(half, half, half)
    return V, T, S.sample_surface(V, T, n, np.random.default_rng(seed))


def _world(solver, gravity=(0, 0, -9.81), mu=0.5, two_free=False):
    V, T, Sp = _cube()
    w = O.OracleWorld(gravity=gravity, solver=solver)
    a = w.add_asset(V, T, Sp)
    if two_free:
        b = w.add_asset(V, T, Sp)
        descs = [S._body(a, S.DYNAMIC, (0, 0, 0), (0, 0, 0, 1), mu, 0.0, (0.3, 0.05, 0), (0.2, -0.1, 0.4)),
                 S._body(b, S.DYNAMIC, (0.02, 0.001, 0.002), (0, 0, 0, 1), mu, 0.0, (-0.2, 0, 0.01), (0, 0.3, 0))]
    else:
        GV, GT = S.box_mesh(0.2, 0.2, 0.01)
        b = w.add_asset(GV, GT, None)
        w.bake(b, 96, 2e-3)
        descs = [S._body(a, S.DYNAMIC, (0, 0, 0.01), (0, 0, 0, 1), mu),
                 S._body(b, S.STATIC, (0, 0, -0.01), (0, 0, 0, 1), mu)]
    bodies = np.zeros((1, 2), S.BODY_DTYPE)
    bodies[0, 0], bodies[0, 1] = descs
    w.add_envs(bodies, np.array([[0, 1]], np.int32))
    return w


def _contacts(xa, n, phi):
    c = np.zeros(len(xa), O.CONTACT_DTYPE)
    c["sample"] = np.arange(len(xa))
    c["xa"], c["n"], c["phi"] = xa, n, phi
    c["xb"] = c["xa"] - c["phi"][:, None] * c["n"]
    return c


def test_one_contact_jacobi_is_gauss_seidel():
    states = []
    for solver in (0, 1):
        w = _world(solver)
        c = _contacts(np.array([[0.01, -0.01, 0.0]]), np.array([[0.1, 0.0, 0.995]]) / np.linalg.norm([0.1, 0, 0.995]),
                      np.array([-2e-5]))
        w.set_contacts(0, c)
        w.substep(1 / 480, 7, detect=False)
        states.append(w.state())
    for x, y in zip(*states):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-13)


@pytest.mark.parametrize("iters", [1, 5, 40])
def test_frictionless_two_bodies_conserve_momentum(iters):
    w = _world(1, gravity=(0, 0, 0), mu=0.0, two_free=True)
    m0 = w.mass(0)[0]
    xa = np.array([[0.01, 0.002, 0.004], [0.01, -0.006, -0.001], [0.0095, 0.004, -0.008]])
    nrm = np.array([[-1.0, 0.05, 0.0], [-1.0, 0.0, 0.1], [-0.98, -0.1, 0.05]])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    c = _contacts(xa, nrm, np.array([-1e-5, -3e-5, 2e-6]))
    p0, q0, v0, w0 = w.state()
    w.set_contacts(0, c)
    w.substep(1 / 240, iters, detect=False)
    p1, q1, v1, w1 = w.state()
    # equal masses; cubes have isotropic inertia, so L = I w + c x m v about the origin
    I = w.mass(0)[2][0, 0]
    P0, P1 = m0 * v0.sum(0), m0 * v1.sum(0)
    L0 = (I * w0 + m0 * np.cross(p0, v0)).sum(0)
    L1 = (I * w1 + m0 * np.cross(p1, v1)).sum(0)
    assert np.abs(v1 - v0).max() > 1e-4          # the contacts acted
    np.testing.assert_allclose(P1, P0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(L1, L0, rtol=0, atol=1e-16)


def test_resting_box_reaches_gauss_seidel_velocities():
    res = []
    for solver, iters in ((0, 400), (1, 6000)):
        w = _world(solver, mu=0.0)
        w.collide()
        w.substep(1 / 240, iters, detect=False)
        res.append(w.state())
    (_, _, vg, wg), (_, _, vj, wj) = res
    # constrained components (normal motion and tilt) agree; frictionless sliding is free
    assert abs(vj[0, 2] - vg[0, 2]) <= 1e-9
    np.testing.assert_allclose(wj[0, :2], wg[0, :2], rtol=0, atol=1e-7)


def test_friction_cone_on_every_row():
    w = _world(1, gravity=(9.81 * math.sin(0.5), 0, -9.81 * math.cos(0.5)), mu=0.3)
    for _ in range(4):
        w.step(4, 32)
        imp = w.impulses(0)
        assert len(imp) > 0
        assert np.all(imp[:, 1] <= imp[:, 2] * imp[:, 0] * (1 + 1e-12) + 1e-18)
