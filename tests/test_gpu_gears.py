"""The gear train on the GPU (three involute spur gears on fixed shafts, 30k triangles and
a 256^3 SDF each, 15k samples on the point gears, two pairs per env and two movable
fixed-axis bodies, so the solve takes its general form) against the FP64 oracle, and
against the gear ratios that involute geometry fixes.

Tolerances as for the other scenes: narrow phase 5e-5 h in phi; normals to (2e-5 +
2^-20 |phi| / h) / |grad| -- each side bakes its own grid and the bakes agree per node to
1e-5 h + 2^-22 |phi|, a gradient component blends node differences over h, so the
gradients differ by up to twice that over h -- except where a sample lies within the pose transform's float32 rounding (1e-4 voxel)
of a cell face: the trilinear gradient jumps across cell faces, and there the two sides may
take either cell (both gears' SDF bodies are rotated and translated, so the transform
rounds at the 1e-5 voxel level); such a flip must stay rare (at most 0.1% of the samples);
reduced contacts identical
where every decision has margin, else agreeing in bulk; identical contacts solved for one
substep to 1e-6 rad; one frame through the whole path to 2e-3 rad (a near-tie resolved
the other way changes a flank contact); the ratios w2/w1 = -z1/z2 and w3/w1 = z1/z3 to 3%
over several frames, in FP32 and with the SDFs stored in FP16.
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
def gears():
    fw = _fw()
    sc = S.gear_scene(n_envs=4, seed=2)
    gw = fw.world_from_scene(sc)
    ow = O.world_from_scene(sc, lazy_bake=True, margin_len=MARGIN_LEN, margin_dot=MARGIN_DOT)
    return sc, gw, ow


def _rot(q):
    x, y, z, w = np.asarray(q, np.float64) / np.linalg.norm(np.asarray(q, np.float64))
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _near_cell_face(gw, sc, env, pair, sdf_asset, tol=1e-4):
    """samples whose grid coordinate (FP64 pose transform of the float32 state) lies within
    tol voxel of a cell face on some axis; bodies of env e are 3e .. 3e + 2 and pair k joins
    bodies k and k + 1"""
    p, q = gw.get_state()[:2]
    a, b = 3 * env + pair, 3 * env + pair + 1
    s = sc.assets[pair].samples.astype(np.float64)
    xw = s @ _rot(q[a]).T + p[a].astype(np.float64)
    xb = (xw - p[b].astype(np.float64)) @ _rot(q[b])
    lo, h = gw.get_sdf(sdf_asset, values=False)[:2]
    u = (xb - lo.astype(np.float64)) / np.float64(h)
    return np.any(np.abs(u - np.round(u)) < tol, axis=1)


def test_narrow_phase_both_pairs(gears):
    sc, gw, ow = gears
    for pair, sdf_asset in ((0, 1), (1, 2)):
        ns = len(sc.assets[pair].samples)
        h = float(gw.get_sdf(sdf_asset, values=False)[1])
        inside = flipped = 0
        for env in range(sc.n_envs):
            phi, nrm = gw.query_pair(env, pair, ns)
            ophi, onrm, ovalid = ow.query_pair(env, pair, ns)
            assert np.array_equal(np.isfinite(phi), ovalid), (env, pair)
            d = np.abs(phi[ovalid] - ophi[ovalid])
            assert np.all(d <= 5e-5 * h), (env, pair, float(d.max() / h))
            near = _near_cell_face(gw, sc, env, pair, sdf_asset)
            dn = np.where(ovalid, np.max(np.abs(nrm - onrm), axis=1), 0.0)
            gtol = 2e-5 + 2.0 ** -20 * np.abs(np.where(ovalid, ophi, 0.0)) / h
            bad = ovalid & (dn > gtol / np.minimum(1.0, np.maximum(ow.last_gnorm, 1e-30)))
            if np.any(bad & ~near):
                i = int(np.flatnonzero(bad & ~near)[0])
                raise AssertionError((env, pair, i, float(dn[i]), float(ow.last_gnorm[i]), float(ophi[i] / h),
                                      nrm[i].tolist(), onrm[i].tolist()))
            assert np.all(np.abs(np.linalg.norm(nrm[ovalid], axis=1) - 1) <= 1e-5)
            inside += int(ovalid.sum())
            flipped += int((bad & near).sum())
        assert inside > 1000, (pair, inside)     # part of the point gear lies in the grid
        assert flipped <= max(2, 1e-3 * inside), (pair, flipped, inside)


def test_collide_per_pair(gears):
    sc, gw, ow = gears
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    gw.collide()
    ow.reset_margins()
    ow.collide()
    for env in range(sc.n_envs):
        gc = gw.get_contacts(env)
        ml, md = ow.margins(env)
        for pair in range(2):
            g = gc[gc["pair"] == pair]
            o = ow.pair_contacts(env, pair)
            assert len(o) > 0, (env, pair)
            if ml >= MARGIN_LEN and md >= MARGIN_DOT:
                assert list(g["sample"]) == list(o["sample"]) and list(g["patch"]) == list(o["patch"])
            else:
                common = len(set(g["sample"]) & set(o["sample"]))
                assert common >= 0.8 * max(len(g), len(o)), (env, pair, common, len(g), len(o))
                assert abs(len(g) - len(o)) <= max(3, 0.15 * len(o)), (env, pair, len(g), len(o))


@pytest.mark.parametrize("shape", [(0, 0), (1, 1)])
def test_solve_identical_contacts_one_substep(gears, shape):
    """Both pairs' contacts given to both sides (float32-rounded), one substep: the general
    sweep form (two movable fixed-axis bodies, pairs in order) at the default shape, and the
    two-body fast rows (one env per warp, pair by pair) at shape (1, 1)."""
    sc, gw, ow = gears
    fw = _fw()
    gw.set_solve_shape(*shape)
    hs = sc.sim.dt / sc.sim.n_substeps
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    ow.collide()
    for env in range(sc.n_envs):
        parts = []
        for pair in range(2):
            o = ow.pair_contacts(env, pair)
            g = np.zeros(len(o), fw.CONTACT_DTYPE)
            g["sample"], g["patch"], g["pair"], g["phi"] = o["sample"], o["patch"], pair, o["phi"]
            g["xa"], g["n"] = o["xa"], o["n"]
            g["xb"] = g["xa"] - g["phi"][:, None] * g["n"]
            same = o.copy()
            same["phi"], same["xa"], same["n"] = g["phi"], g["xa"], g["n"]
            same["xb"] = same["xa"] - same["phi"][:, None] * same["n"]
            ow.set_pair_contacts(env, pair, same)
            parts.append(g)
        gw.set_contacts(env, np.concatenate(parts))
    gw.substep(hs, sc.sim.n_iters, detect=False)
    ow.substep(hs, sc.sim.n_iters, detect=False)
    gw.set_solve_shape(0, 0)
    gp, gq, gv, gom = gw.get_state()
    op, oq, ov, oom = ow.state()
    for i in range(len(gp)):
        assert np.linalg.norm(gp[i] - op[i]) <= 1e-6, (i, shape, gp[i], op[i])
        assert _rot_angle(gq[i].astype(np.float64), oq[i]) <= 1e-6, (i, shape, gq[i], oq[i])
    assert np.max(np.abs(gom - oom)) <= 1e-4 * max(1.0, float(np.max(np.abs(oom))))


def test_one_frame_against_the_oracle(gears):
    sc, gw, ow = gears
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    gw.step(sc.sim.n_substeps, sc.sim.n_iters)
    ow.step(sc.sim.n_substeps, sc.sim.n_iters)
    gp, gq, gv, gom = gw.get_state()
    op, oq, ov, oom = ow.state()
    np.testing.assert_allclose(gp, op, rtol=0, atol=1e-7)      # fixed shafts, kinematic driver
    assert np.all(gv == 0) and np.all(gom[:, :2] == 0)
    for i in range(len(gp)):
        assert _rot_angle(gq[i].astype(np.float64), oq[i]) <= 2e-3, (i, gq[i], oq[i])


@pytest.mark.parametrize("fp16", [False, True])
def test_train_turns_at_the_gear_ratios(fp16):
    fw = _fw()
    sc = S.gear_scene(n_envs=32, seed=5)
    w = fw.world_from_scene(sc, fp16=fp16)
    z1, z2, z3 = S.GEAR_TEETH
    om2, om3 = [], []
    for _ in range(8):
        w.step(sc.sim.n_substeps, sc.sim.n_iters)
        om = w.get_state()[3]
        om2.append(om[1::3, 2])
        om3.append(om[2::3, 2])
    np.testing.assert_allclose(np.mean(om2, axis=0), -2.0 * z1 / z2, rtol=0.03)
    np.testing.assert_allclose(np.mean(om3, axis=0), 2.0 * z1 / z3, rtol=0.03)
    w.close()
