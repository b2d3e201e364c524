"""Piles of nuts on the GPU: up to 8 free bodies per env coupled through 28 pairs (every
nut against the plate and against every other nut), the general Gauss-Seidel form, and
the query kernel's broad phase (items of a pair whose bounding spheres are apart by more
than the contact offset plus two voxels are skipped) against the FP64 oracle, which has
no broad phase.

Tolerances as for the other scenes: contact sets per pair identical where the decisions
have margin and in bulk otherwise, so a skipped pair must have no contacts on the oracle's
side either; identical contacts solved for one substep to 1e-6 m / rad; a frame of the
stacks to 2e-4 m / 2e-3 rad.
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


@pytest.fixture(scope="module")
def stacks():
    fw = _fw()
    sc = S.pile_scene(n_envs=6, seed=3, n_nuts=7, mode="stacks")
    gw = fw.world_from_scene(sc)
    ow = O.world_from_scene(sc, lazy_bake=True, margin_len=MARGIN_LEN, margin_dot=MARGIN_DOT)
    return sc, gw, ow


def test_collide_per_pair_and_broad_phase(stacks):
    sc, gw, ow = stacks
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    gw.collide()
    ow.reset_margins()
    ow.collide()
    pairs = sc.groups[0].pairs
    r_nut = float(np.linalg.norm(sc.assets[0].verts, axis=1).max())
    far = near = 0
    for env in range(sc.n_envs):
        gc = gw.get_contacts(env)
        ml, md = ow.margins(env)
        for k, (i, j) in enumerate(pairs):
            g = gc[gc["pair"] == k]
            o = ow.pair_contacts(env, k)
            if j < 7 and np.linalg.norm(p[8 * env + i] - p[8 * env + j]) > 2 * r_nut + 3e-3:
                assert len(g) == 0 and len(o) == 0, (env, k)   # skipped by the broad phase
                far += 1
                continue
            if len(o) == 0:
                assert len(g) == 0
                continue
            near += 1
            if ml >= MARGIN_LEN and md >= MARGIN_DOT:
                assert list(g["sample"]) == list(o["sample"]) and list(g["patch"]) == list(o["patch"])
            else:
                common = len(set(g["sample"]) & set(o["sample"]))
                assert common >= 0.8 * max(len(g), len(o)), (env, k, common, len(g), len(o))
    assert far > 20 and near > 20, (far, near)


@pytest.mark.parametrize("shape", [(0, 0), (1, 1)])
def test_solve_identical_contacts_one_substep(stacks, shape):
    """Identical contacts, one substep: the default shape (two envs per warp: the general
    form, lane 0 of an env's lanes over full rows) and one env per warp (the two-body fast
    rows, pair by pair with four lanes per pair)."""
    sc, gw, ow = stacks
    fw = _fw()
    gw.set_solve_shape(*shape)
    hs = sc.sim.dt / sc.sim.n_substeps
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    ow.collide()
    n_pairs = len(sc.groups[0].pairs)
    for env in range(sc.n_envs):
        parts = []
        for k in range(n_pairs):
            o = ow.pair_contacts(env, k)
            g = np.zeros(len(o), fw.CONTACT_DTYPE)
            g["sample"], g["patch"], g["pair"], g["phi"] = o["sample"], o["patch"], k, o["phi"]
            g["xa"], g["n"] = o["xa"], o["n"]
            g["xb"] = g["xa"] - g["phi"][:, None] * g["n"]
            same = o.copy()
            same["phi"], same["xa"], same["n"] = g["phi"], g["xa"], g["n"]
            same["xb"] = same["xa"] - same["phi"][:, None] * same["n"]
            ow.set_pair_contacts(env, k, same)
            parts.append(g)
        gw.set_contacts(env, np.concatenate(parts))
    gw.substep(hs, sc.sim.n_iters, detect=False)
    ow.substep(hs, sc.sim.n_iters, detect=False)
    gw.set_solve_shape(0, 0)
    gp, gq = gw.get_state()[:2]
    op, oq = ow.state()[:2]
    for i in range(len(gp)):
        assert np.linalg.norm(gp[i] - op[i]) <= 1e-6, (i, shape, gp[i], op[i])
        assert _rot_angle(gq[i].astype(np.float64), oq[i]) <= 1e-6, (i, shape, gq[i], oq[i])


def test_one_frame_of_stacks(stacks):
    sc, gw, ow = stacks
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    gw.step(sc.sim.n_substeps, sc.sim.n_iters)
    ow.step(sc.sim.n_substeps, sc.sim.n_iters)
    gp, gq = gw.get_state()[:2]
    op, oq = ow.state()[:2]
    for i in range(len(gp)):
        assert np.linalg.norm(gp[i] - op[i]) <= 2e-4, (i, gp[i], op[i])
        assert _rot_angle(gq[i].astype(np.float64), oq[i]) <= 2e-3, (i, gq[i], oq[i])


def test_dropped_pile_comes_to_rest_on_the_plate():
    fw = _fw()
    sc = S.pile_scene(n_envs=16, seed=5, n_nuts=7, mode="drop")
    w = fw.world_from_scene(sc)
    for _ in range(150):
        w.step(sc.sim.n_substeps, sc.sim.n_iters)
    p, q, v, om = w.get_state()
    nuts = [i for i in range(len(p)) if i % 8 != 7]
    assert np.all(np.isfinite(p))
    on = np.all(np.abs(p[nuts, :2]) < 0.06, axis=1)                  # over the plate (a nut may roll off)
    assert on.mean() >= 0.9, on.mean()
    assert np.all(p[nuts][on, 2] > 0.0)                               # none fell through the plate
    speed = np.linalg.norm(v[nuts][on], axis=1)
    assert np.median(speed) < 5e-3, np.median(speed)
    w.close()
