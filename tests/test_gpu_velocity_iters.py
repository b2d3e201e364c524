"""Velocity iterations (n_vel_iters bias-free sweeps after the integration) on the GPU
against the oracle on identical contacts, one substep: the fast form (one movable body),
the general form (two movable bodies) and the Jacobi solver, to 1e-6 m / 1e-6 rad as for
the position sweeps."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


def _fw():
    from paper_2205_03532_b300 import fw
    return fw


def _rot_angle(q1, q2):
    d = abs(float(np.dot(q1 / np.linalg.norm(q1), q2 / np.linalg.norm(q2))))
    return 2 * math.acos(min(1.0, d))


def _peg():
    sc = S.peg_in_hole_scene(n_envs=32, seed=12)
    b = sc.groups[0].bodies
    rng = np.random.default_rng(12)
    b["pos"][:, 0, 2] = 12.5e-3 + rng.uniform(-4e-3, 0.2e-3, len(b))
    b["pos"][:, 0, :2] = rng.uniform(-0.09e-3, 0.09e-3, (len(b), 2))
    return sc


def _two_cubes():
    """envs of two dynamic cubes, the upper one resting tilted on the lower one"""
    V, T = S.box_mesh(0.01, 0.01, 0.01)
    Sp = S.sample_surface(V, T, 900, np.random.default_rng(3))
    a = S.Asset("cube", V, T, Sp, 7800.0)
    b = S.Asset("cube_sdf", V, T, None, 7800.0, sdf_res=48, sdf_pad=3e-3)
    rng = np.random.default_rng(4)
    bodies = np.zeros((8, 2), S.BODY_DTYPE)
    for e in range(8):
        q = S.quat_mul(S.quat_axis_angle([0, 0, 1], rng.uniform(0, 1)), S.quat_axis_angle([1, 0, 0], rng.uniform(-0.2, 0.2)))
        bodies[e, 0] = S._body(0, S.DYNAMIC, (0.0, 0.004, 0.0203), q, 0.4, 0.0, (0, 0, -0.3), (0.5, -1, 0))
        bodies[e, 1] = S._body(1, S.DYNAMIC, (0, 0, 0), (0, 0, 0, 1), 0.4, 0.02, (0.01, 0, 0.05))
    sim = S.SimParams(n_substeps=4, n_iters=16)
    return S.Scene("two_cubes", [a, b], [S.EnvGroup(bodies, np.array([[0, 1]], np.int32))], sim)


@pytest.mark.parametrize("scene,solver", [("peg", 0), ("cubes", 0), ("peg", 1)])
def test_velocity_iterations_identical_contacts(scene, solver):
    fw = _fw()
    sc = _peg() if scene == "peg" else _two_cubes()
    gw = fw.world_from_scene(sc, n_vel_iters=3, solver=solver)
    ow = O.world_from_scene(sc, n_vel_iters=3, solver=solver)
    hs = sc.sim.dt / sc.sim.n_substeps
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    ow.collide()
    n = 0
    for env in range(sc.n_envs):
        oc, _, _ = ow.contacts(env)
        gc = np.zeros(len(oc), fw.CONTACT_DTYPE)
        gc["sample"], gc["patch"], gc["phi"] = oc["sample"], oc["patch"], oc["phi"]
        gc["xa"], gc["n"] = oc["xa"], oc["n"]
        gc["xb"] = gc["xa"] - gc["phi"][:, None] * gc["n"]
        same = oc.copy()
        same["phi"], same["xa"], same["n"] = gc["phi"], gc["xa"], gc["n"]
        same["xb"] = same["xa"] - same["phi"][:, None] * same["n"]
        gw.set_contacts(env, gc)
        ow.set_contacts(env, same)
        n += len(oc)
    assert n > 0
    iters = 16 if solver == 0 else 64
    gw.substep(hs, iters, detect=False)
    ow.substep(hs, iters, detect=False)
    gp, gq, gv, gom = gw.get_state()
    op, oq, ov, oom = ow.state()
    for i in range(len(gp)):
        assert np.linalg.norm(gp[i] - op[i]) <= 1e-6, (i, gp[i], op[i])
        assert _rot_angle(gq[i].astype(np.float64), oq[i]) <= 1e-6, (i, gq[i], oq[i])
    assert np.max(np.abs(gv - ov)) <= 1e-4 * max(1.0, float(np.max(np.abs(ov))))
    assert np.max(np.abs(gom - oom)) <= 1e-4 * max(1.0, float(np.max(np.abs(oom))))
    gw.close()
