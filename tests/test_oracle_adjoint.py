"""The oracle's reverse mode (differentiable rollout with the discrete decisions held fixed).

Pins, all on the CPU:
  * a recorded rollout is the oracle's plain forward (same contacts, same formulas);
  * the adjoint equals central finite differences of the taped replay for every input:
    initial position, orientation (rotation vector), linear and angular velocity, the
    dynamic body's mass (inertia scaled at fixed geometry) and the pair's friction
    coefficient -- in contact with a static hole and with a moving kinematic slab;
  * free flight: d p_T / d p_0 = I, d p_T / d v_0 = T I, d v_T / d v_0 = I exactly.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


def _peg_scene(n_envs=2, seed=3, mu=0.5):
    sc = S.peg_in_hole_scene(n_envs=n_envs, seed=seed, clearance_mm=0.1, mu=mu, n_substeps=8, n_iters=8)
    b = sc.groups[0].bodies
    rng = np.random.default_rng(seed)
    # partly inserted, tilted, moving down and sideways: contacts on the hole's wall and floor
    b["pos"][:, 0, 2] = 12.5e-3 - rng.uniform(1e-3, 3e-3, len(b))
    b["pos"][:, 0, :2] = rng.uniform(-0.08e-3, 0.08e-3, (len(b), 2))
    b["linvel"][:, 0] = [0.004, -0.003, -0.02]
    b["angvel"][:, 0] = [0.3, -0.2, 0.5]
    for e in range(len(b)):
        t = np.deg2rad(rng.uniform(-0.4, 0.4, 2))
        b["quat"][e, 0] = S.quat_mul(S.quat_axis_angle([1, 0, 0], t[0]), S.quat_axis_angle([0, 1, 0], t[1]))
    return sc


def _slab_scene():
    """a cube resting on a kinematic slab that slides and turns: friction drags it"""
    V, T = S.box_mesh(0.01, 0.01, 0.01)
    Sp = S.sample_surface(V, T, 600, np.random.default_rng(2))
    GV, GT = S.box_mesh(0.1, 0.1, 0.01)
    cube = S.Asset("cube", V, T, Sp, 7800.0)
    slab = S.Asset("slab", GV, GT, None, 7800.0, 48, 2e-3)
    b = np.zeros((1, 2), S.BODY_DTYPE)
    q = S.quat_axis_angle([0.3, 1, 0.2], 0.02)
    b[0, 0] = S._body(0, S.DYNAMIC, (0.001, -0.002, 0.00998), q, 0.6, 0.0, (0.01, 0, -0.01), (0.1, 0.2, 0.3))
    b[0, 1] = S._body(1, S.KINEMATIC, (0, 0, -0.01), (0, 0, 0, 1), 0.6, 0.0, (0.05, 0.02, 0), (0, 0, 0.4))
    sim = S.SimParams(n_substeps=6, n_iters=10)
    return S.Scene("slab", [cube, slab], [S.EnvGroup(b, np.array([[0, 1]], np.int32))], sim)


def _world(sc):
    return O.world_from_scene(sc, lazy_bake=True)


def test_recorded_rollout_is_the_plain_forward():
    sc = _peg_scene()
    a, b = _world(sc), _world(sc)
    a.step(sc.sim.n_substeps, sc.sim.n_iters)
    b.diff_record(sc.sim.n_substeps, sc.sim.n_iters)
    sa, sb = a.state(), b.state()
    for x, y in zip(sa, sb):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-12)
    t = b.get_tape()
    assert len(t["c_rec"]) > 20 * sc.sim.n_substeps       # in contact all along


def _rot(theta, q0):
    ang = np.linalg.norm(theta)
    if ang == 0:
        return np.asarray(q0, float)
    return S.quat_mul(S.quat_axis_angle(theta / ang, ang), q0)


def _check_fd(sc, body, pair, seed):
    w = _world(sc)
    x0 = [a.copy() for a in w.state()]
    w.diff_record(sc.sim.n_substeps, sc.sim.n_iters)
    w.set_state(*x0)
    rng = np.random.default_rng(seed)
    nb = len(x0[0])
    g = [rng.normal(size=(nb, k)) for k in (3, 4, 3, 3)]
    g[0] *= 1e3   # weight positions (m) against velocities so that every term matters
    adj = w.diff_adjoint(*g)

    def loss_at(xs):
        w.set_state(*xs)
        w.diff_replay()
        return sum(float(np.sum(gi * si)) for gi, si in zip(g, w.state()))

    def central(f, h):
        """Richardson-extrapolated central difference: error O(h^4)"""
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        return (4 * d2 - d1) / 3

    def shifted(idx, k, t):
        xs = [a.copy() for a in x0]
        xs[idx][body, k] += t
        return loss_at(xs)

    checks = []
    # position, velocity, angular velocity
    for comp, (idx, h) in {"pos": (0, 1e-7), "linvel": (2, 1e-6), "angvel": (3, 1e-5)}.items():
        for k in range(3):
            checks.append((f"{comp}[{k}]", adj[comp][body, k], central(lambda t: shifted(idx, k, t), h)))
    # orientation through a rotation vector: q(theta) = exp(theta) q0
    q0 = x0[1][body]
    for k in range(3):
        e = np.zeros(3); e[k] = 1.0
        dq = 0.5 * S.quat_mul(np.array([e[0], e[1], e[2], 0.0]), q0)
        an = float(np.dot(adj["quat"][body], dq))

        def rotated(t):
            xs = [a.copy() for a in x0]
            xs[1][body] = _rot(t * e, q0)
            return loss_at(xs)
        checks.append((f"rot[{k}]", an, central(rotated, 1e-6)))
    # mass (inertia scaled with it) and the pair's friction coefficient
    mass = w.body_mass(body)
    for name, setter, v0, h in (("mass", lambda v: w.set_body_mass(body, v), mass, 1e-6 * mass),
                                ("mu", lambda v: w.set_pair_mu(pair, v), w.pair_mu(pair), 1e-6)):
        def param(t):
            setter(v0 + t)
            return loss_at(x0)
        d = central(param, h)
        setter(v0)
        checks.append((name, adj[name][body if name == "mass" else pair], d))
    scale = max(abs(c[2]) for c in checks)
    for name, a, d in checks:
        assert abs(a - d) <= 2e-6 * max(abs(d), 1e-3 * scale), (name, a, d)
    return checks


def test_adjoint_matches_central_differences_in_the_hole():
    checks = _check_fd(_peg_scene(n_envs=1, seed=5), body=0, pair=0, seed=1)
    assert abs(dict((c[0], c[2]) for c in checks)["mu"]) > 0      # friction matters here


def test_adjoint_matches_central_differences_on_a_kinematic_slab():
    checks = _check_fd(_slab_scene(), body=0, pair=0, seed=2)
    assert abs(dict((c[0], c[2]) for c in checks)["mu"]) > 0


def test_free_flight_closed_form():
    sc = _peg_scene(n_envs=1, seed=1)
    b = sc.groups[0].bodies
    b["pos"][0, 0, 2] = 0.2      # far above the box: no contact
    w = _world(sc)
    x0 = [a.copy() for a in w.state()]
    w.diff_record(sc.sim.n_substeps, sc.sim.n_iters)
    assert len(w.get_tape()["c_rec"]) == 0
    w.set_state(*x0)
    nb = len(x0[0])
    T = sc.sim.dt
    for k in range(3):
        gp = np.zeros((nb, 3)); gp[0, k] = 1.0
        z3, z4 = np.zeros((nb, 3)), np.zeros((nb, 4))
        adj = w.diff_adjoint(gp, z4, z3, z3)
        e = np.eye(3)[k]
        np.testing.assert_allclose(adj["pos"][0], e, atol=1e-12)
        np.testing.assert_allclose(adj["linvel"][0], T * e, atol=1e-12)
        assert abs(adj["mass"][0]) < 1e-12
        adj = w.diff_adjoint(z3, z4, gp, z3)
        np.testing.assert_allclose(adj["linvel"][0], e, atol=1e-12)
        np.testing.assert_allclose(adj["pos"][0], 0, atol=1e-12)
