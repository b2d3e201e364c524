"""Pins of the oracle's substep (Gauss-Seidel contact solve with Coulomb friction and
substepped integration; Sec. III-B) against closed forms and physical invariants."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S

RNG = np.random.default_rng(0)


def _cube(half=0.01, n_samples=600, seed=0):
    V, T = S.box_mesh(half, half, half)
    return V, T, S.sample_surface(V, T, n_samples, np.random.default_rng(seed))


def _ground(half_xy=0.1, half_z=0.01):
    return S.box_mesh(half_xy, half_xy, half_z)


def _desc(asset, btype, pos, quat=(0, 0, 0, 1), mu=0.5, mass=0.0, v=(0, 0, 0), w=(0, 0, 0),
          axis=(0, 0, 1), force=(0, 0, 0), torque=(0, 0, 0)):
    return S._body(asset, btype, pos, quat, mu, mass, v, w, axis, force, torque)


def _one_env(w, descs, pairs):
    bodies = np.zeros((1, len(descs)), S.BODY_DTYPE)
    for i, d in enumerate(descs):
        bodies[0, i] = d
    w.add_envs(bodies, np.array(pairs, np.int32).reshape(-1, 2))


# ---------------------------------------------------------------- integration without contact
def test_free_fall_closed_form():
    V, T, Sp = _cube()
    w = O.OracleWorld(gravity=(0, 0, -9.81))
    a = w.add_asset(V, T, Sp)
    _one_env(w, [_desc(a, S.DYNAMIC, (0, 0, 1.0), v=(0.1, 0, 0.5))], [])
    hs, K = 1.0 / 240, 37
    for _ in range(K):
        w.substep(hs, 8)
    p, q, v, _ = w.state()
    vx0, g = float(np.float32(0.1)), 9.81   # body descriptors carry float32; the config is float64
    # semi-implicit Euler: v_k = v0 - g h k, z_k = z0 + v0 h k - g h^2 k (k + 1) / 2
    assert p[0, 2] == pytest.approx(1.0 + 0.5 * hs * K - g * hs * hs * K * (K + 1) / 2, abs=1e-13)
    assert p[0, 0] == pytest.approx(vx0 * hs * K, abs=1e-15)
    assert v[0, 2] == pytest.approx(0.5 - g * hs * K, abs=1e-13)


def test_torque_free_isotropic_spin_closed_form():
    V, T, Sp = _cube()
    w = O.OracleWorld(gravity=(0, 0, 0))
    a = w.add_asset(V, T, Sp)
    axis = np.array([1.0, 2.0, -0.5]) / np.linalg.norm([1.0, 2.0, -0.5])
    wmag = 7.3
    _one_env(w, [_desc(a, S.DYNAMIC, (0, 0, 0), w=tuple(axis * wmag))], [])
    hs, K = 1.0 / 480, 200
    for _ in range(K):
        w.substep(hs, 4)
    _, q, _, om = w.state()
    w0 = (axis * wmag).astype(np.float32).astype(np.float64)   # as stored in the descriptor
    axis, wmag = w0 / np.linalg.norm(w0), np.linalg.norm(w0)
    # an isotropic body has no gyroscopic torque: omega is constant
    np.testing.assert_allclose(om[0], w0, atol=1e-12)
    # q <- normalize(q + h/2 (omega, 0) q) turns by exactly 2 atan(|omega| h / 2) per step
    ang = 2 * math.atan2(np.linalg.norm(q[0, :3]), q[0, 3])
    assert ang == pytest.approx(K * 2 * math.atan(wmag * hs / 2), abs=1e-11)
    np.testing.assert_allclose(q[0, :3] / np.linalg.norm(q[0, :3]), axis, atol=1e-12)


def _quat_mat(q):
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _free_spin(V, T, w0, quat, K, t_end):
    """oracle: one free body, no gravity, no contact, K substeps over t_end; (q, omega, I_b)"""
    w = O.OracleWorld(gravity=(0, 0, 0))
    a = w.add_asset(V, T, S.sample_surface(V, T, 50, np.random.default_rng(0)))
    _one_env(w, [_desc(a, S.DYNAMIC, (0, 0, 0), quat=quat, w=tuple(w0))], [])
    for _ in range(K):
        w.substep(t_end / K, 1)
    _, q, _, om = w.state()
    return q[0], om[0], w.mass(a)[2]


def test_torque_free_anisotropic_spin_converges_to_euler_equations():
    """The gyroscopic term of the external-force step (omega += hs I_w^-1 (tau - omega x
    I_w omega)): a 10 x 20 x 40 mm box spinning about a non-principal axis, against Euler's
    equations of a torque-free rigid body integrated to 1e-12 by scipy (DOP853) with the
    box's analytic inertia.  The substep is first order, so the error halves with the step;
    without the term (or with its sign flipped) omega would stay constant (or turn the wrong
    way) and the error would be O(1) at any step: 1.41 rad/s here against <= 0.036."""
    from scipy.integrate import solve_ivp
    hx, hy, hz = 0.005, 0.01, 0.02
    V, T = S.box_mesh(hx, hy, hz)
    w0 = np.array([3.0, 1.0, 2.0])
    t_end = 1.0
    m = 7800.0 * (2 * hx) * (2 * hy) * (2 * hz)
    Ib = np.diag([m / 12 * ((2 * hy) ** 2 + (2 * hz) ** 2), m / 12 * ((2 * hx) ** 2 + (2 * hz) ** 2),
                  m / 12 * ((2 * hx) ** 2 + (2 * hy) ** 2)])

    def rhs(_, y):   # world form: dR/dt = [omega]x R, d(I_w omega)/dt = 0
        R, om = y[:9].reshape(3, 3), y[9:]
        Iw = R @ Ib @ R.T
        W = np.array([[0, -om[2], om[1]], [om[2], 0, -om[0]], [-om[1], om[0], 0]])
        return np.concatenate([(W @ R).ravel(), -np.linalg.solve(Iw, np.cross(om, Iw @ om))])

    w0f = w0.astype(np.float32).astype(np.float64)   # as stored in the descriptor
    sol = solve_ivp(rhs, (0, t_end), np.concatenate([np.eye(3).ravel(), w0f]), method="DOP853", rtol=1e-12,
                    atol=1e-14)
    om_ref = sol.y[9:, -1]
    L0 = Ib @ w0f
    assert np.linalg.norm(om_ref - w0f) > 1.0            # the term matters: omega turns by O(1)
    err, drift = [], []
    for K in (200, 400):
        q, om, I = _free_spin(V, T, w0, (0, 0, 0, 1), K, t_end)
        R = _quat_mat(q)
        err.append(np.linalg.norm(om - om_ref))
        drift.append(np.linalg.norm(R @ I @ R.T @ om - L0))
    assert err[0] < 0.025 and drift[0] < 6e-3 * np.linalg.norm(L0)
    assert 1.8 < err[0] / err[1] < 2.2                  # first order in the step
    assert 1.8 < drift[0] / drift[1] < 2.2              # world angular momentum: conserved to O(h)


def test_spin_about_a_principal_axis_is_steady():
    """omega along a principal axis of an anisotropic box (its long axis, the box turned by
    a general rotation): omega x I_w omega = 0, so omega stays constant."""
    V, T = S.box_mesh(0.005, 0.01, 0.02)
    quat = np.array([0.3, -0.5, 0.2, 0.79])
    quat /= np.linalg.norm(quat)
    q32 = quat.astype(np.float32).astype(np.float64)
    axis = _quat_mat(q32 / np.linalg.norm(q32)) @ np.array([0.0, 0.0, 1.0])
    w0 = 6.0 * axis
    q, om, _ = _free_spin(V, T, w0, tuple(quat), 300, 0.5)
    w0f = w0.astype(np.float32).astype(np.float64)
    # the float32 descriptor leaves omega off the axis by ~1e-7 relative; the off-axis part
    # then nutates, at that size
    np.testing.assert_allclose(om, w0f, atol=1e-5 * np.linalg.norm(w0f))


def test_kinematic_body_follows_prescribed_velocity():
    V, T, Sp = _cube()
    w = O.OracleWorld(gravity=(0, 0, -9.81))
    a = w.add_asset(V, T, Sp)
    _one_env(w, [_desc(a, S.KINEMATIC, (0.1, 0, 0), v=(0.2, -0.1, 0.05))], [])
    for _ in range(50):
        w.substep(0.004, 4)
    p, _, v, _ = w.state()
    np.testing.assert_allclose(p[0], [0.1 + 0.2 * 0.2, -0.1 * 0.2, 0.05 * 0.2], atol=1e-14)
    np.testing.assert_allclose(v[0], [0.2, -0.1, 0.05], atol=0)


def test_fixed_axis_body_spins_about_its_axis_only():
    V, T = S.cylinder_mesh(0.01, 0.005, 24)
    w = O.OracleWorld(gravity=(0, 0, -9.81))
    a = w.add_asset(V, T, S.sample_surface(V, T, 100, np.random.default_rng(1)))
    ax = np.array([0.0, 0.6, 0.8])
    _one_env(w, [_desc(a, S.FIXED_AXIS, (0.01, 0.02, 0.03), axis=tuple(ax), torque=(1e-3, 2e-3, 3e-3))], [])
    m, com, I = w.mass(a)
    ax = ax.astype(np.float32).astype(np.float64)
    ax /= np.linalg.norm(ax)                                   # the body's stored axis
    for _ in range(100):
        w.substep(0.002, 4)
    p, q, v, om = w.state()
    np.testing.assert_allclose(v[0], 0, atol=0)
    np.testing.assert_allclose(np.cross(om[0], ax), 0, atol=1e-14 * np.linalg.norm(om[0]))
    # angular acceleration about the axis: (a . tau) / (a^T I_w a), I_w rotating about a
    R0 = np.eye(3)
    Iaa = ax @ (R0 @ I @ R0.T) @ ax
    tau = np.array([1e-3, 2e-3, 3e-3], np.float32).astype(np.float64)
    w_expect = 100 * 0.002 * (ax @ tau) / Iaa
    assert om[0] @ ax == pytest.approx(w_expect, rel=1e-9)


# ---------------------------------------------------------------- contact
def _cube_on_ground(mu=0.5, gravity=(0, 0, -9.81), gz_offset=0.0, n_samples=600):
    V, T, Sp = _cube(n_samples=n_samples)
    GV, GT = _ground(0.2, 0.01)
    w = O.OracleWorld(gravity=gravity)
    a = w.add_asset(V, T, Sp)
    g = w.add_asset(GV, GT, None)
    w.bake(g, 96, 2e-3)
    _one_env(w, [_desc(a, S.DYNAMIC, (0, 0, 0.01 + gz_offset), mu=mu),
                 _desc(g, S.STATIC, (0, 0, -0.01), mu=mu)], [(0, 1)])
    return w


def test_resting_box_does_not_drift():
    w = _cube_on_ground()
    p0 = w.state()[0][0].copy()
    for _ in range(120):
        w.step(4, 16)
    p, q, v, om = w.state()
    assert abs(p[0, 2] - p0[2]) <= 1e-6
    assert np.linalg.norm(p[0, :2] - p0[:2]) <= 1e-6
    assert np.linalg.norm(v[0]) <= 1e-4 and np.linalg.norm(om[0]) <= 1e-3
    c, _, _ = w.contacts(0)
    assert 4 <= len(c) <= 7                       # one patch: deepest + direction extremes
    assert len(np.unique(c["patch"])) == 1


def test_friction_cone_holds_on_every_row():
    w = _cube_on_ground(mu=0.3, gravity=(9.81 * math.sin(0.5), 0, -9.81 * math.cos(0.5)))
    for _ in range(5):
        w.step(4, 16)
        imp = w.impulses(0)
        assert len(imp) > 0
        assert np.all(imp[:, 0] >= 0.0)
        assert np.all(imp[:, 1] <= imp[:, 2] * imp[:, 0] * (1 + 1e-9) + 1e-18)
        # sliding: at least one row is on the cone boundary
        assert np.any(imp[:, 1] >= imp[:, 2] * imp[:, 0] * (1 - 1e-9))


@pytest.mark.parametrize("theta_deg, mu", [(10.0, 0.3), (25.0, 0.3), (30.0, 0.1)])
def test_inclined_plane_stick_or_slide(theta_deg, mu):
    th = math.radians(theta_deg)
    g = 9.81
    w = _cube_on_ground(mu=mu, gravity=(g * math.sin(th), 0, -g * math.cos(th)))
    frames = []
    for f in range(16):   # the slide stays on the 0.4 m ground for this long
        w.step(4, 32)
        p, _, v, _ = w.state()
        frames.append((p[0].copy(), v[0].copy()))
    if math.tan(th) <= mu:
        assert abs(frames[-1][0][0]) <= 1e-5          # sticks
    else:
        a_exp = g * (math.sin(th) - mu * math.cos(th))
        a_meas = (frames[-1][1][0] - frames[3][1][0]) / (12 / 60.0)
        assert a_meas == pytest.approx(a_exp, rel=0.02)
        assert abs(frames[-1][0][2] - 0.01) <= 1e-5   # stays on the plane


def test_frictionless_collision_conserves_momentum():
    V, T, Sp = _cube(n_samples=800)
    w = O.OracleWorld(gravity=(0, 0, 0))
    a = w.add_asset(V, T, Sp)
    b = w.add_asset(V, T, None)
    w.bake(b, 48, 3e-3)
    q = S.quat_mul(S.quat_axis_angle([0, 0, 1], 0.3), S.quat_axis_angle([1, 0, 0], 0.2))
    _one_env(w, [_desc(a, S.DYNAMIC, (0.0, 0.004, 0.0205), quat=q, mu=0.0, v=(0, 0, -0.3), w=(0.5, -1, 0)),
                 _desc(b, S.DYNAMIC, (0, 0, 0), mu=0.0, mass=0.02, v=(0.01, 0, 0.05))], [(0, 1)])
    m, _, I = w.mass(a)
    mb = float(np.float32(0.02))
    masses = [m, mb]
    inertias = [I, I * mb / m]

    def momenta():
        p, qq, v, om = w.state()
        P = sum(masses[i] * v[i] for i in range(2))
        L = sum(inertias[i] @ om[i] + masses[i] * np.cross(p[i], v[i]) for i in range(2))
        return P, L

    P0, L0 = momenta()
    touched = 0
    for _ in range(20):
        w.step(4, 16)
        c, _, _ = w.contacts(0)
        touched += len(c) > 0
        P, L = momenta()
        np.testing.assert_allclose(P, P0, rtol=0, atol=1e-15)
        np.testing.assert_allclose(L, L0, rtol=0, atol=1e-16)
    assert touched > 0
    # and the bodies did exchange momentum
    _, _, v, _ = w.state()
    assert abs(v[1, 2] - 0.05) > 1e-3


def _rotate_scene_world(Rq, tilt_q, mu, gravity):
    """Cube dropped tilted onto a ground slab; the whole scene (poses, gravity) turned by Rq."""
    V, T, Sp = _cube(n_samples=500)
    GV, GT = _ground(0.1, 0.01)
    Rm = _qm(Rq)
    w = O.OracleWorld(gravity=tuple(Rm @ np.asarray(gravity)))
    a = w.add_asset(V, T, Sp)
    g = w.add_asset(GV, GT, None)
    w.bake(g, 64, 2e-3)
    cube_p = Rm @ np.array([0.001, -0.002, 0.0125])
    ground_p = Rm @ np.array([0.0, 0.0, -0.01])
    _one_env(w, [_desc(a, S.DYNAMIC, tuple(cube_p), quat=tuple(S.quat_mul(Rq, tilt_q)), mu=mu),
                 _desc(g, S.STATIC, tuple(ground_p), quat=tuple(Rq), mu=mu)], [(0, 1)])
    return w


def _qm(q):
    x, y, z, w_ = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w_), 2 * (x * z + y * w_)],
                     [2 * (x * y + z * w_), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w_)],
                     [2 * (x * z - y * w_), 2 * (y * z + x * w_), 1 - 2 * (x * x + y * y)]])


def test_frictionless_drop_is_rotation_equivariant():
    """Without friction no rule depends on the world axes, so turning the whole scene
    turns the result.  This pins the frame transforms (R_A s + p_A, R_B^T (x - p_B),
    R_B g / |g|) and the quaternion conventions.  Rotations by a quarter turn about a
    world axis keep every float32 input exact."""
    tilt = S.quat_mul(S.quat_axis_angle([1, 0, 0], 0.15), S.quat_axis_angle([0, 1, 0], -0.1))
    ref = _rotate_scene_world(np.array([0, 0, 0, 1.0]), tilt, 0.0, (0, 0, -9.81))
    Rq = S.quat_axis_angle([1, 0, 0], math.pi / 2)
    Rq = np.round(Rq * 2 ** 20) / 2 ** 20
    Rq /= np.linalg.norm(Rq)
    rot = _rotate_scene_world(Rq, tilt, 0.0, (0, 0, -9.81))
    Rm = _qm(Rq)
    touched = 0
    for _ in range(12):
        ref.step(4, 16)
        rot.step(4, 16)
        touched += len(ref.contacts(0)[0]) > 0
        p0, q0, v0, w0 = ref.state()
        p1, q1, v1, w1 = rot.state()
        np.testing.assert_allclose(p1[0], Rm @ p0[0], atol=2e-8)
        np.testing.assert_allclose(v1[0], Rm @ v0[0], atol=2e-6)
        np.testing.assert_allclose(w1[0], Rm @ w0[0], atol=2e-4)
        np.testing.assert_allclose(_qm(q1[0]), Rm @ _qm(q0[0]), atol=2e-6)
    assert touched >= 3


def test_penetration_is_pushed_out_by_the_bias():
    """A cube started 0.2 mm into the ground: the bias baumgarte * phi / hs must push it
    out (never deeper), converging to the surface."""
    w = _cube_on_ground(gz_offset=-2e-4, mu=0.5)
    z0 = 0.01 - 2e-4
    zs = []
    for f in range(60):
        w.step(4, 16)
        zs.append(w.state()[0][0, 2])
    zs = np.array(zs)
    assert np.all(zs >= z0)                        # never sinks deeper
    assert np.all(np.diff(zs[:5]) > 0)             # recovers while the depth is large
    assert np.all(np.abs(zs[20:] - 0.01) <= 2e-6)  # and settles on the surface
