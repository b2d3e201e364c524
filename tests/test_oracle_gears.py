"""The gear train (three involute spur gears on fixed parallel shafts, the first one driven,
the last one loaded) through the oracle, pinned by the geometry of involute gearing rather
than by the oracle's own code:

  * the meshes are closed, consistently wound 2-manifolds near the triangle count asked for;
  * in the conjugate starting position (a tooth of one gear centred in a gap of the next)
    the flanks clear each other by about half the backlash, so no candidate lies deeper
    than the jitter allows;
  * once the teeth are loaded the train turns at the gear ratios: for involute profiles in
    mesh the angular velocities satisfy w2 / w1 = -z1 / z2 and w3 / w2 = -z2 / z3 exactly
    (constant ratio is the defining property of conjugate profiles), so over several frames
    the driven gears turn at -4/3 and +1 rad/s under the 2 rad/s drive, up to the play
    the backlash leaves;
  * fixed-axis bodies: the centre of mass never moves and the spin stays on the shaft.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


def test_gear_meshes_are_closed_and_near_the_triangle_target():
    for a in S.gear_assets(tri_target=30000, n_samples=10, sdf_res=16):
        assert S.edge_manifold_check(a.tris), a.name
        assert S.signed_volume(a.verts, a.tris) > 0
        assert 0.8 * 30000 <= len(a.tris) <= 1.2 * 30000, (a.name, len(a.tris))


@pytest.fixture(scope="module")
def train():
    sc = S.gear_scene(n_envs=2, seed=1, tri_target=8000, n_samples=3000, sdf_res=128)
    w = O.world_from_scene(sc, lazy_bake=True)
    w.collide()
    return sc, w


def test_conjugate_start_has_clearance(train):
    sc, w = train
    jitter = 0.2 * 0.1e-3          # the scene's per-gear jitter bound (arc length)
    for env in range(sc.n_envs):
        for pair in range(2):
            c = w.pair_contacts(env, pair)
            assert len(c) > 0, (env, pair)
            # half the backlash minus two jitters, minus the SDF's interpolation error
            assert c["phi"].min() >= 0.5 * 0.1e-3 - 2 * jitter - 2e-5, (env, pair, c["phi"].min())


def test_train_turns_at_the_gear_ratios(train):
    sc, w = train
    z1, z2, z3 = S.GEAR_TEETH
    om2, om3 = [], []
    p0 = w.state()[0].copy()
    for _ in range(6):
        w.step(sc.sim.n_substeps, sc.sim.n_iters)
        p, q, v, om = w.state()
        np.testing.assert_array_equal(v, 0.0)
        np.testing.assert_array_equal(om[:, :2], 0.0)
        np.testing.assert_allclose(p, p0, rtol=0, atol=1e-15)
        om2.append(om[1::3, 2])
        om3.append(om[2::3, 2])
    drive = 2.0
    m2, m3 = np.mean(om2, axis=0), np.mean(om3, axis=0)
    np.testing.assert_allclose(m2, -drive * z1 / z2, rtol=0.03)
    np.testing.assert_allclose(m3, drive * z1 / z3, rtol=0.03)
