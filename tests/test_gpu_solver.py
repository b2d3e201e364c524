"""GPU solver paths against the FP64 oracle on identical contacts, and invariants.

The solve kernel has a fast form (at most one movable body per env; rows written from
that body's side) and a general form (several movable bodies).  Each is checked after one
substep on contacts computed by the oracle and rounded to float32 for both sides:
positions within 1e-6 m, orientations within 1e-6 rad."""
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


def _pair_worlds(descs, assets, pairs, **cfg):
    """GPU and oracle worlds with one env of the given bodies."""
    fw = _fw()
    gw = fw.World(**cfg)
    ow = O.OracleWorld(**cfg)
    for V, T, Sp, res, pad in assets:
        a = gw.add_mesh_asset(V, T, Sp)
        b = ow.add_asset(V, T, Sp)
        assert a == b
        if res:
            gw.bake_sdf(a, res, pad)
            ow.bake(b, res, pad)
    bodies = np.zeros((1, len(descs)), S.BODY_DTYPE)
    for i, d in enumerate(descs):
        bodies[0, i] = d
    gw.add_env_bodies(bodies, np.array(pairs, np.int32))
    ow.add_envs(bodies, np.array(pairs, np.int32))
    return gw, ow


def _solve_same_contacts(gw, ow, hs, n_iters, keep=None):
    fw = _fw()
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    ow.collide()
    oc, _, _ = ow.contacts(0)
    assert len(oc) > 0
    if keep is not None:      # the deepest `keep` contacts only
        oc = oc[np.argsort(oc["phi"], kind="stable")[:keep]]
    gc = np.zeros(len(oc), fw.CONTACT_DTYPE)
    gc["sample"], gc["patch"], gc["phi"] = oc["sample"], oc["patch"], oc["phi"]
    gc["xa"], gc["n"] = oc["xa"], oc["n"]
    gc["xb"] = gc["xa"] - gc["phi"][:, None] * gc["n"]
    same = oc.copy()
    same["phi"], same["xa"], same["n"] = gc["phi"], gc["xa"], gc["n"]
    same["xb"] = same["xa"] - same["phi"][:, None] * same["n"]
    gw.set_contacts(0, gc)
    ow.set_contacts(0, same)
    gw.substep(hs, n_iters, detect=False)
    ow.substep(hs, n_iters, detect=False)
    gs, os_ = gw.get_state(), ow.state()
    for i in range(len(gs[0])):
        assert np.linalg.norm(gs[0][i] - os_[0][i]) <= 1e-6, (i, gs[0][i], os_[0][i])
        assert _rot_angle(gs[1][i].astype(np.float64), os_[1][i]) <= 1e-6
        assert np.linalg.norm(gs[2][i] - os_[2][i]) <= 1e-4 * max(1.0, np.linalg.norm(os_[2][i]))
    return len(oc)


def _cube(half=0.01, n=700, seed=0):
    V, T = S.box_mesh(half, half, half)
    return V, T, S.sample_surface(V, T, n, np.random.default_rng(seed))


def test_general_path_two_dynamic_bodies():
    V, T, Sp = _cube()
    q = S.quat_mul(S.quat_axis_angle([0, 0, 1], 0.3), S.quat_axis_angle([1, 0, 0], 0.2))
    descs = [S._body(0, S.DYNAMIC, (0.0, 0.004, 0.0203), q, 0.4, 0.0, (0, 0, -0.3), (0.5, -1, 0)),
             S._body(1, S.DYNAMIC, (0, 0, 0), (0, 0, 0, 1), 0.4, 0.02, (0.01, 0, 0.05))]
    gw, ow = _pair_worlds(descs, [(V, T, Sp, None, 0), (V, T, None, 48, 3e-3)], [(0, 1)], gravity=(0, 0, -9.81))
    assert _solve_same_contacts(gw, ow, 1 / 240, 16) > 0


def test_fast_path_with_the_sdf_body_moving():
    """The point body is static, the SDF body is dynamic: rows are written from the SDF
    body's side (negated directions)."""
    GV, GT = S.box_mesh(0.05, 0.05, 0.005)
    Gs = S.sample_surface(GV, GT, 6000, np.random.default_rng(1))
    V, T, _ = _cube()
    tilt = S.quat_mul(S.quat_axis_angle([1, 0, 0], 0.1), S.quat_axis_angle([0, 1, 0], 0.05))
    descs = [S._body(0, S.STATIC, (0, 0, -0.005), (0, 0, 0, 1), 0.6),
             S._body(1, S.DYNAMIC, (0.002, 0.001, 0.0105), tilt, 0.6, 0.0, (0.05, 0, -0.1), (0, 0.5, 0))]
    gw, ow = _pair_worlds(descs, [(GV, GT, Gs, None, 0), (V, T, None, 48, 3e-3)], [(0, 1)])
    assert _solve_same_contacts(gw, ow, 1 / 240, 16) > 0


def test_fast_path_kinematic_partner_velocity_enters_the_rows():
    """A cube resting on a kinematic slab that moves sideways: friction must drag it."""
    V, T, Sp = _cube()
    GV, GT = S.box_mesh(0.1, 0.1, 0.01)
    descs = [S._body(0, S.DYNAMIC, (0, 0, 0.01), (0, 0, 0, 1), 0.5),
             S._body(1, S.KINEMATIC, (0, 0, -0.01), (0, 0, 0, 1), 0.5, 0.0, (0.2, 0, 0), (0, 0, 0.3))]
    gw, ow = _pair_worlds(descs, [(V, T, Sp, None, 0), (GV, GT, None, 64, 2e-3)], [(0, 1)])
    _solve_same_contacts(gw, ow, 1 / 240, 16)
    v = gw.get_state()[2]
    assert v[0, 0] > 1e-3          # dragged along by friction
    np.testing.assert_allclose(v[1], [0.2, 0, 0], atol=0)


@pytest.mark.parametrize("keep", [1, 2, 3])
def test_fast_path_with_one_two_three_contacts(keep):
    """Fewest rows: one contact (the fast sweep pads it with an all-zero row), two (each
    row's neighbour is the other), three.  A tilted cube pressed onto a kinematic slab."""
    V, T, Sp = _cube()
    GV, GT = S.box_mesh(0.1, 0.1, 0.01)
    tilt = S.quat_mul(S.quat_axis_angle([1, 0, 0], 0.15), S.quat_axis_angle([0, 1, 0], 0.1))
    descs = [S._body(0, S.DYNAMIC, (0, 0, 0.0117), tilt, 0.5, 0.0, (0.05, 0.02, -0.2), (0.3, -0.2, 0.4)),
             S._body(1, S.KINEMATIC, (0, 0, -0.01), (0, 0, 0, 1), 0.5, 0.0, (0.1, 0, 0), (0, 0, 0.3))]
    gw, ow = _pair_worlds(descs, [(V, T, Sp, None, 0), (GV, GT, None, 64, 2e-3)], [(0, 1)])
    assert _solve_same_contacts(gw, ow, 1 / 240, 16, keep=keep) == keep


def test_envs_without_contacts_beside_envs_in_contact():
    """Envs with no contact share warps with envs in contact (every solve shape); the
    solve's masked steps for them must leave their free flight exact, frame after frame,
    whatever the shared memory held before (the reduction kernel leaves all-ones words)."""
    fw = _fw()
    sc = S.peg_in_hole_scene(n_envs=64, seed=11)
    b = sc.groups[0].bodies
    b["pos"][:, 0, 2] = 12.5e-3 - 1e-3              # partly inserted: in contact
    b["pos"][1::2, 0, 2] = 1.0                        # far above the box: free flight
    b["linvel"][1::2, 0] = [0.01, -0.02, 0.3]
    b["angvel"][1::2, 0] = [0.5, -1.0, 2.0]
    hs = np.float32(np.float32(sc.sim.dt) / sc.sim.n_substeps)
    for shape in [(1, 1), (2, 1), (4, 2), (8, 4)]:
        w = fw.world_from_scene(sc)
        w.set_solve_shape(*shape)
        v0 = w.get_state()[2].copy()
        K = 3 * sc.sim.n_substeps
        for _ in range(3):
            w.step(sc.sim.n_substeps, sc.sim.n_iters)
        p, q, v, om = w.get_state()
        assert np.all(np.isfinite(p)) and np.all(np.isfinite(q)), shape
        free = np.arange(2, len(p), 4)                # the pegs of the odd envs
        g = np.float32(9.81)
        assert np.allclose(v[free, 2], v0[free, 2] - g * hs * K, atol=1e-5), shape
        assert np.array_equal(v[free, :2], v0[free, :2]), shape
        assert np.all(np.isfinite(om)), shape
        w.close()


def test_free_fall_on_gpu_matches_closed_form():
    fw = _fw()
    V, T, Sp = _cube()
    w = fw.World()
    a = w.add_mesh_asset(V, T, Sp)
    b = np.zeros((1, 1), S.BODY_DTYPE)
    b[0, 0] = S._body(a, S.DYNAMIC, (0, 0, 1.0), (0, 0, 0, 1), 0.5, 0.0, (0.1, 0, 0.5))
    w.add_env_bodies(b, np.zeros((0, 2), np.int32))
    K = 40
    for _ in range(K // 4):
        w.step(4, 8)
    p, _, v, _ = w.get_state()
    hs = np.float32(1 / 60) / 4
    g = 9.81
    z = 1.0 + 0.5 * hs * K - g * hs * hs * K * (K + 1) / 2
    assert abs(p[0, 2] - z) <= 2e-6 and abs(v[0, 2] - (0.5 - g * hs * K)) <= 1e-5


def test_frictionless_two_body_momentum_on_gpu():
    fw = _fw()
    V, T, Sp = _cube(n=800)
    w = fw.World(gravity=(0, 0, 0))
    a = w.add_mesh_asset(V, T, Sp)
    bb = w.add_mesh_asset(V, T, None)
    w.bake_sdf(bb, 48, 3e-3)
    q = S.quat_mul(S.quat_axis_angle([0, 0, 1], 0.3), S.quat_axis_angle([1, 0, 0], 0.2))
    b = np.zeros((1, 2), S.BODY_DTYPE)
    b[0, 0] = S._body(a, S.DYNAMIC, (0.0, 0.004, 0.0205), q, 0.0, 0.0, (0, 0, -0.3), (0.5, -1, 0))
    b[0, 1] = S._body(bb, S.DYNAMIC, (0, 0, 0), (0, 0, 0, 1), 0.0, 0.02, (0.01, 0, 0.05))
    w.add_env_bodies(b, np.array([[0, 1]], np.int32))
    m, _, I = w.get_mass(a)
    mb = float(np.float32(0.02))
    masses, inertias = [m, mb], [I, I * mb / m]

    def momenta():
        p, _, v, om = w.get_state()
        P = sum(masses[i] * v[i].astype(np.float64) for i in range(2))
        L = sum(inertias[i] @ om[i] + masses[i] * np.cross(p[i].astype(np.float64), v[i]) for i in range(2))
        return P, L

    P0, L0 = momenta()
    for _ in range(20):
        w.step(4, 16)
    P, L = momenta()
    np.testing.assert_allclose(P, P0, atol=2e-8)     # float32 rounding of ~1e-3 kg m/s
    np.testing.assert_allclose(L, L0, atol=2e-10)
    assert abs(w.get_state()[2][1, 2] - 0.05) > 1e-3  # they did collide


def test_solve_shapes_give_bit_identical_results():
    """Envs sharing a warp (2 or 4 per warp) and blocks of several warps run the same
    arithmetic per env as one env per warp: states agree bit for bit.  Fast-form envs
    (one dynamic cube on a static slab) and envs of two movable bodies (two dynamic cubes)
    are interleaved so that warps hold both kinds, and the env count leaves ragged warps
    and blocks.  The two-movable envs run the general form when they share a warp and the
    two-body fast rows with a warp each (shapes (1, w)): bit for bit within each of the
    two, and to float32 rounding between them."""
    fw = _fw()
    V, T, Sp = _cube(n=900)
    GV, GT = S.box_mesh(0.05, 0.05, 0.005)
    w = fw.World()
    a = w.add_mesh_asset(V, T, Sp)
    slab = w.add_mesh_asset(GV, GT, None)
    w.bake_sdf(slab, 64, 2e-3)
    cb = w.add_mesh_asset(V, T, None)
    w.bake_sdf(cb, 48, 3e-3)
    rng = np.random.default_rng(5)

    def fast_group(n):
        b = np.zeros((n, 2), S.BODY_DTYPE)
        for e in range(n):
            q = S.quat_mul(S.quat_axis_angle([1, 0, 0], rng.uniform(-0.2, 0.2)),
                           S.quat_axis_angle([0, 0, 1], rng.uniform(0, 1)))
            b[e, 0] = S._body(a, S.DYNAMIC, (rng.uniform(-0.01, 0.01), 0, 0.0148), q, 0.5, 0.0,
                              (rng.uniform(-0.2, 0.2), 0, -0.1), (0, rng.uniform(-2, 2), 0))
            b[e, 1] = S._body(slab, S.STATIC, (0, 0, 0), (0, 0, 0, 1), 0.5)
        return b

    def general_group(n):
        b = np.zeros((n, 2), S.BODY_DTYPE)
        for e in range(n):
            q = S.quat_axis_angle([0, 0, 1], rng.uniform(0, 1))
            b[e, 0] = S._body(a, S.DYNAMIC, (0.0, 0.002, 0.0203), q, 0.4, 0.0, (0, 0, -0.3), (0.5, -1, 0))
            b[e, 1] = S._body(cb, S.DYNAMIC, (0, 0, 0), (0, 0, 0, 1), 0.4, 0.02, (0.01, 0, 0.05))
        return b

    for g in (fast_group(5), general_group(3), fast_group(4), general_group(1), fast_group(6)):
        w.add_env_bodies(g, np.array([[0, 1]], np.int32))
    s0 = [x.copy() for x in w.get_state()]
    results = {}
    for shape in [(1, 1), (1, 4), (2, 1), (2, 3), (4, 1), (4, 4), (8, 1), (8, 2)]:
        w.set_solve_shape(*shape)
        eff = w.solve_shape()               # lowered when the blocks would not fit in shared memory
        assert eff[0] == shape[0] and 1 <= eff[1] <= shape[1]
        w.set_state(*s0)
        for _ in range(3):
            w.step(4, 16)
        results[shape] = w.get_state()
    ref, refg = results[(1, 1)], results[(2, 1)]
    assert np.abs(ref[0] - s0[0]).max() > 1e-5          # the bodies did move
    general = np.zeros(len(ref[0]), bool)              # the bodies of the two-movable envs
    for e in (5, 6, 7, 12):
        general[2 * e:2 * e + 2] = True
    for shape, st in results.items():
        for x, y, yg in zip(st, ref, refg):
            np.testing.assert_array_equal(x[~general], y[~general], err_msg=str(shape))
            np.testing.assert_array_equal(x[general], (y if shape[0] == 1 else yg)[general], err_msg=str(shape))
            # the two forms sum in different float32 orders; over 12 substeps of two cubes in
            # contact the difference grows to ~3e-5 (angular velocity); their per-substep parity
            # with the FP64 oracle (1e-6) is checked in the gear and pile tests
            np.testing.assert_allclose(y[general], yg[general], rtol=1e-2, atol=1e-4, err_msg=str(shape))
    w.set_solve_shape(0, 0)
    assert w.solve_shape() == (2, 1)                     # 19 envs: two per warp, one warp per block
    with pytest.raises(fw.FwError):
        w.set_solve_shape(3, 1)


def test_detect_shapes_give_identical_contacts_and_the_autotuner_keeps_them():
    """Every detection launch shape (query threads 128 / 256 / 512, reduction warps 2 / 4 /
    8) gives the same contacts bit for bit; the autotuner picks one of them and leaves the
    state and the contacts as they were."""
    fw = _fw()
    sc = S.nut_bolt_scene(n_envs=24, seed=5)
    w = fw.world_from_scene(sc)
    for _ in range(2):
        w.step(sc.sim.n_substeps, sc.sim.n_iters)
    s0 = [a.copy() for a in w.get_state()]
    ref = None
    for qt in (256, 128, 512):
        for rw in (4, 2, 8):
            w.set_detect_shape(qt, rw)
            assert w.detect_shape() == (qt, rw)
            w.collide()
            got = [w.get_contacts(e) for e in range(sc.n_envs)]
            if ref is None:
                ref = got
                assert sum(len(c) for c in ref) > 1000
            else:
                for a, b in zip(ref, got):
                    assert a.tobytes() == b.tobytes(), (qt, rw)
    qt, rw, ms = w.autotune_detect(trials=2)
    assert qt in (128, 256, 512) and rw in (2, 4, 8) and ms > 0
    assert w.detect_shape() == (qt, rw)
    for a, b in zip(ref, [w.get_contacts(e) for e in range(sc.n_envs)]):
        assert a.tobytes() == b.tobytes()
    for a, b in zip(s0, w.get_state()):
        np.testing.assert_array_equal(a, b)
    with pytest.raises(fw.FwError):
        w.set_detect_shape(64, 4)
    w.close()
