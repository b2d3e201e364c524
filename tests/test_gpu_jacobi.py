"""The weighted Jacobi solver on the GPU (solver = 1: every contact's block update from the
sweep-start velocities, all taken with weight 1 / active contacts; one movable body per
env) against the oracle's Jacobi on the same contacts.

Tolerances: the GPU sums the contacts' velocity changes over a group's lanes (a different
order from the oracle's, and from one solve shape to another), so identical contacts
agree to 1e-6 m / 1e-6 rad after one substep, as for Gauss-Seidel, and shapes agree to
the same bound rather than bit for bit; a frame through the whole path agrees to 1e-5 on
envs whose detection decisions have margin.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S

MARGIN_LEN, MARGIN_DOT = 1e-7, 1e-6


def _fw():
    from paper_2205_03532_b300 import fw
    return fw


def _rot_angle(q1, q2):
    d = abs(float(np.dot(q1 / np.linalg.norm(q1), q2 / np.linalg.norm(q2))))
    return 2 * math.acos(min(1.0, d))


def _peg(n_envs=64, seed=7):
    sc = S.peg_in_hole_scene(n_envs=n_envs, seed=seed)
    b = sc.groups[0].bodies
    rng = np.random.default_rng(seed)
    b["pos"][:, 0, 2] = 12.5e-3 + rng.uniform(-4e-3, 0.3e-3, len(b))
    b["pos"][:, 0, :2] = rng.uniform(-0.09e-3, 0.09e-3, (len(b), 2))
    return sc


def _close(gs, os_, pos_tol, rot_tol, bodies):
    for i in bodies:
        assert np.linalg.norm(gs[0][i] - os_[0][i]) <= pos_tol, (i, gs[0][i], os_[0][i])
        assert _rot_angle(gs[1][i].astype(np.float64), os_[1][i]) <= rot_tol, (i, gs[1][i], os_[1][i])


@pytest.mark.parametrize("scene", ["peg", "nut"])
def test_identical_contacts_one_substep(scene):
    fw = _fw()
    sc = _peg() if scene == "peg" else S.nut_bolt_scene(n_envs=4, seed=1)
    gw = fw.world_from_scene(sc, solver=1)
    ow = O.world_from_scene(sc, lazy_bake=True, solver=1)
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
    gw.substep(hs, 64, detect=False)
    ow.substep(hs, 64, detect=False)
    gs, os_ = gw.get_state(), ow.state()
    _close(gs, os_, 1e-6, 1e-6, range(len(gs[0])))
    assert np.max(np.abs(gs[2] - os_[2])) <= 1e-4 * max(1.0, float(np.max(np.abs(os_[2]))))
    gw.close()


def test_frame_against_the_oracle():
    fw = _fw()
    sc = _peg(n_envs=32, seed=3)
    gw = fw.world_from_scene(sc, solver=1)
    ow = O.world_from_scene(sc, solver=1, margin_len=MARGIN_LEN, margin_dot=MARGIN_DOT)
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    ow.reset_margins()
    gw.step(sc.sim.n_substeps, 64)
    ow.step(sc.sim.n_substeps, 64)
    gs, os_ = gw.get_state(), ow.state()
    ok = 0
    for env in range(sc.n_envs):
        ml, md = ow.margins(env)
        if ml >= MARGIN_LEN and md >= MARGIN_DOT:
            _close(gs, os_, 1e-5, 1e-5, [2 * env])
            ok += 1
        else:
            _close(gs, os_, 2e-4, 2e-3, [2 * env])
    assert ok >= 1
    gw.close()


def test_solve_shapes_agree():
    """one substep of 64 sweeps from the same state: the shapes differ only in the order of
    the per-lane sums"""
    fw = _fw()
    sc = S.nut_bolt_scene(n_envs=64, seed=2)
    outs = []
    for shape in ((1, 1), (2, 1), (4, 2), (8, 4)):
        w = fw.world_from_scene(sc, solver=1)
        w.set_solve_shape(*shape)
        w.substep(sc.sim.dt / sc.sim.n_substeps, 64)
        outs.append(w.get_state())
        w.close()
    for o in outs[1:]:
        _close(o, [x.astype(np.float64) for x in outs[0]], 1e-6, 1e-6, range(0, len(o[0]), 2))


def test_refusals():
    fw = _fw()
    sc = S.gear_scene(n_envs=1, seed=0, tri_target=4000, n_samples=500, sdf_res=32)
    with pytest.raises(fw.FwError):
        fw.world_from_scene(sc, solver=1)          # two movable gears in one env
    w = fw.world_from_scene(_peg(n_envs=2), solver=1)
    with pytest.raises(fw.FwError):
        w.record_rollout(2, 4)                     # no adjoint of the Jacobi solver
    w.close()
