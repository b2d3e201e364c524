"""GPU adjoint of the differentiable rollout (reverse mode with the decisions taped).

* the recorded rollout moves the bodies as the regular fw_step does;
* short rollout (8 substeps of 1/960 s, 8 sweeps; a pressed, jammed peg), where the
  gradient is well conditioned: the GPU adjoint equals the FP64 oracle's adjoint on the
  GPU's own tape to 1e-3 in every env, and Richardson-extrapolated central differences of
  the taped rollout to 1e-3 (90th percentile over envs); the differences are evaluated in
  FP64 by the oracle replaying the GPU's tape (the same frozen function without float32
  rounding noise), with steps that move the peg by about 1 um;
* the full differentiable peg workload (one frame of 32 substeps x 8 sweeps): the
  gradient of a jammed, pressed peg over a whole frame is ill conditioned -- moving the
  initial positions by 1e-9 m (one float32 ulp) changes the exact FP64 adjoint by up to
  about 1e-2 -- so there each env's GPU error must stay within a few times that
  measured sensitivity;
* the GPU adjoint against float32 central differences of its own replay, a gross-error
  check only (median within 5e-2): the rounding noise of the final float32 state bounds
  what such a difference resolves;
* the torch.autograd.Function gives the ABI's gradients through a pose loss.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


def _fw():
    from paper_2205_03532_b300 import fw
    return fw


def _world(n_envs, n_substeps, seed=2):
    fw = _fw()
    sc, tp, tq = S.diff_peg_scene(n_envs=n_envs, seed=seed, n_substeps=n_substeps, n_iters=8)
    sc.sim.dt = n_substeps / 960.0 if n_substeps < 32 else sc.sim.dt   # substeps of 1/960 s or 1/1920 s
    w = fw.world_from_scene(sc)
    return sc, w, [a.copy() for a in w.get_state()]


@pytest.fixture(scope="module")
def diff_world():
    return _world(32, 8)


@pytest.fixture(scope="module")
def frame_world():
    return _world(64, 32)


def _rand_g(nb, seed):
    rng = np.random.default_rng(seed)
    g = [rng.normal(size=(nb, k)).astype(np.float32) for k in (3, 4, 3, 3)]
    g[0] *= 1e3
    return g


def test_recorded_rollout_moves_like_step(diff_world):
    fw = _fw()
    sc, w, x0 = diff_world
    w.set_state(*x0)
    w.record_rollout(sc.sim.n_substeps, sc.sim.n_iters)
    rec = w.get_state()
    w2 = fw.world_from_scene(sc)
    w2.step(sc.sim.n_substeps, sc.sim.n_iters)
    ref = w2.get_state()
    pegs = slice(0, None, 2)
    dp = np.abs(rec[0][pegs] - ref[0][pegs]).max()
    assert dp <= 2e-6, dp            # float32 rounding of two orderings of the same sweep
    assert np.abs(rec[0][pegs] - x0[0][pegs]).max() > 1e-5
    t = w.get_tape()
    assert len(t["c_rec"]) > 10 * sc.sim.n_substeps * sc.n_envs


def _oracle_on_gpu_tape(sc, w, x0, g):
    tape = w.get_tape()
    tape["hs"] = sc.sim.dt / sc.sim.n_substeps
    ow = O.world_from_scene(sc, lazy_bake=True)
    ow.set_state(*[a.astype(np.float64) for a in x0])
    ow.set_tape(tape)
    return ow, ow.diff_adjoint(*[a.astype(np.float64) for a in g])


def _rel_err(gpu, orc, sc, pegs):
    out = {}
    for name, k, idx in (("pos", 0, pegs), ("quat", 1, pegs), ("linvel", 2, pegs), ("angvel", 3, pegs),
                         ("mass", 4, pegs), ("mu", 5, np.arange(sc.n_envs))):
        a, b = gpu[k][idx].astype(np.float64), orc[name][idx]
        if a.ndim == 1:
            a, b = a[:, None], b[:, None]
        nrm = np.linalg.norm(b, axis=1)
        out[name] = np.linalg.norm(a - b, axis=1) / np.maximum(nrm, 1e-3 * nrm.max())
    return out


def test_gpu_adjoint_matches_oracle_on_the_same_tape(diff_world):
    sc, w, x0 = diff_world
    w.set_state(*x0)
    w.record_rollout(sc.sim.n_substeps, sc.sim.n_iters)
    nb = len(x0[0])
    g = _rand_g(nb, 3)
    gpu = w.adjoint_rollout(*g)
    _, orc = _oracle_on_gpu_tape(sc, w, x0, g)
    errs = _rel_err(gpu, orc, sc, np.arange(0, nb, 2))
    print("\nshort rollout, GPU vs oracle adjoint on the GPU tape (median / max relative error): " +
          ", ".join(f"{n} {np.median(e):.1e}/{e.max():.1e}" for n, e in errs.items()))
    for name, e in errs.items():
        assert np.quantile(e, 0.95) <= 1e-3 and e.max() <= 5e-3, (name, float(e.max()))


def test_step_fwd_ckpt_and_step_bwd_are_record_and_adjoint(diff_world):
    """The frame-step names of the interface run the same operations: same final state,
    same adjoints, bit for bit."""
    sc, w, x0 = diff_world
    nb = len(x0[0])
    g = _rand_g(nb, 5)
    w.set_state(*x0)
    w.record_rollout(sc.sim.n_substeps, sc.sim.n_iters)
    s1 = [a.copy() for a in w.get_state()]
    a1 = w.adjoint_rollout(*g)
    w.set_state(*x0)
    w.step_fwd_ckpt(sc.sim.n_substeps, sc.sim.n_iters)
    s2 = w.get_state()
    a2 = w.step_bwd(*g)
    for x, y in zip(s1, s2):
        np.testing.assert_array_equal(x, y)
    for x, y in zip(a1, a2):
        np.testing.assert_array_equal(x, y)


def test_full_frame_adjoint_within_the_problems_conditioning(frame_world):
    sc, w, x0 = frame_world
    w.set_state(*x0)
    w.record_rollout(sc.sim.n_substeps, sc.sim.n_iters)
    nb = len(x0[0])
    pegs = np.arange(0, nb, 2)
    g = _rand_g(nb, 6)
    gpu = w.adjoint_rollout(*g)
    ow, orc = _oracle_on_gpu_tape(sc, w, x0, g)
    errs = _rel_err(gpu, orc, sc, pegs)
    # sensitivity of the exact adjoint to float32-sized changes of the initial positions
    rng = np.random.default_rng(7)
    sens = {k: np.zeros_like(v) for k, v in errs.items()}
    for _ in range(2):
        xs = [a.astype(np.float64) for a in x0]
        xs[0][pegs] += 1e-9 * rng.normal(size=(len(pegs), 3))
        ow.set_state(*xs)
        alt = ow.diff_adjoint(*[a.astype(np.float64) for a in g])
        alt_as_gpu = (alt["pos"], alt["quat"], alt["linvel"], alt["angvel"], alt["mass"], alt["mu"])
        for k, v in _rel_err(alt_as_gpu, orc, sc, pegs).items():
            sens[k] = np.maximum(sens[k], v)
    print("\nframe of 32 substeps, GPU vs oracle (median / max) and the oracle's own change under "
          "1e-9 m (max): " + ", ".join(f"{n} {np.median(e):.1e}/{e.max():.1e} ({sens[n].max():.1e})"
                                       for n, e in errs.items()))
    for name, e in errs.items():
        assert np.median(e) <= 1e-3, (name, float(np.median(e)))
        assert np.all(e <= 5.0 * sens[name] + 2e-4), (name, float((e - 5.0 * sens[name]).max()))


def _rot(theta, q0):
    ang = np.linalg.norm(theta)
    return np.asarray(q0, float) if ang == 0 else S.quat_mul(S.quat_axis_angle(theta / ang, ang), q0)


def _fd_cases(sc, x0, adj, loss_per_env, set_mass, set_mu, pegs, steps):
    """Richardson central differences for every input of every peg env"""
    mass0 = sc.groups[0].bodies["mass"][:, 0].astype(np.float64)
    mu0 = sc.groups[0].bodies["mu"][:, 0].astype(np.float64)

    def central(f, h):
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        return (4 * d2 - d1) / 3

    def shifted(idx, k, t):
        xs = [a.copy() for a in x0]
        xs[idx][pegs, k] += t
        return loss_per_env(xs)

    def rotated(k, t):
        xs = [a.copy() for a in x0]
        e = np.eye(3)[k]
        for b in pegs:
            xs[1][b] = _rot(t * e, x0[1][b])
        return loss_per_env(xs)

    def with_mass(t):
        set_mass(mass0 * (1.0 + t))
        out = loss_per_env(x0)
        set_mass(mass0)
        return out

    def with_mu(t):
        set_mu(mu0 + t)
        out = loss_per_env(x0)
        set_mu(mu0)
        return out

    cases = []
    for comp, idx in (("pos", 0), ("linvel", 2), ("angvel", 3)):
        for k in range(3):
            cases.append((f"{comp}[{k}]", adj[idx][pegs, k].astype(np.float64),
                          central(lambda t: shifted(idx, k, t), steps[comp])))
    for k in range(3):
        e = np.eye(3)[k]
        an = np.array([np.dot(adj[1][b], 0.5 * S.quat_mul(np.array([e[0], e[1], e[2], 0.0]), x0[1][b]))
                       for b in pegs])
        cases.append((f"rot[{k}]", an, central(lambda t: rotated(k, t), steps["rot"])))
    cases.append(("mass", adj[4][pegs].astype(np.float64) * mass0, central(with_mass, steps["mass"])))
    cases.append(("mu", adj[5].astype(np.float64), central(with_mu, steps["mu"])))
    out = []
    for name, an, fd in cases:
        err = np.abs(an - fd) / np.maximum(np.abs(fd), 1e-2 * np.abs(fd).max())
        out.append((name, float(np.median(err)), float(np.quantile(err, 0.9)), float(err.max())))
    return out


def test_gpu_adjoint_matches_central_differences(diff_world):
    """differences of the taped rollout, evaluated in FP64 by the oracle on the GPU's tape"""
    sc, w, x0 = diff_world
    nb = len(x0[0])
    pegs = np.arange(0, nb, 2)
    w.set_state(*x0)
    w.record_rollout(sc.sim.n_substeps, sc.sim.n_iters)
    tape = w.get_tape()
    tape["hs"] = sc.sim.dt / sc.sim.n_substeps
    g = _rand_g(nb, 4)
    adj = w.adjoint_rollout(*g)
    ow = O.world_from_scene(sc, lazy_bake=True)
    ow.set_tape(tape)
    g64 = [a.astype(np.float64) for a in g]

    def loss_per_env(xs):
        ow.set_state(*[a.astype(np.float64) for a in xs])
        ow.diff_replay()
        return sum((gi * si).sum(axis=1) for gi, si in zip(g64, ow.state()))[pegs]

    def set_mass(m):
        for e, b in enumerate(pegs):
            ow.set_body_mass(int(b), float(m[e]))

    def set_mu(mu):
        for pi in range(sc.n_envs):
            ow.set_pair_mu(pi, float(mu[pi]))

    x64 = [a.astype(np.float64) for a in x0]
    steps = dict(pos=1e-6, linvel=6e-5, angvel=5e-3, rot=4e-5, mass=1e-5, mu=1e-5)
    report = _fd_cases(sc, x64, adj, loss_per_env, set_mass, set_mu, pegs, steps)
    print("\nGPU adjoint vs FP64 central differences of the taped rollout (median / 90th pct / max): " +
          ", ".join(f"{n} {a:.1e}/{b:.1e}/{c:.1e}" for n, a, b, c in report))
    for name, med, p90, mx in report:
        assert p90 <= 1e-3 and med <= 1e-4 and mx <= 1e-2, (name, med, p90, mx)


def test_gpu_adjoint_consistent_with_its_float32_replay(diff_world):
    sc, w, x0 = diff_world
    nb = len(x0[0])
    pegs = np.arange(0, nb, 2)
    w.set_state(*x0)
    w.record_rollout(sc.sim.n_substeps, sc.sim.n_iters)
    g = _rand_g(nb, 5)
    adj = w.adjoint_rollout(*g)

    def loss_per_env(xs):
        w.set_state(*xs)
        w.replay_rollout()
        return sum((gi.astype(np.float64) * si).sum(axis=1) for gi, si in zip(g, w.get_state()))[pegs]

    def set_mass(m):
        full = np.full(nb, -1.0, np.float32)
        full[pegs] = m
        w.set_body_params(mass=full)

    def set_mu(mu):
        w.set_body_params(mu=np.asarray(mu, np.float32))

    steps = dict(pos=4e-6, linvel=2.4e-4, angvel=2e-2, rot=1.6e-4, mass=1e-4, mu=1e-4)
    report = _fd_cases(sc, x0, adj, loss_per_env, set_mass, set_mu, pegs, steps)
    w.set_state(*x0)
    print("\nGPU adjoint vs float32 central differences of its replay (median / 90th pct / max): " +
          ", ".join(f"{n} {a:.1e}/{b:.1e}/{c:.1e}" for n, a, b, c in report))
    for name, med, p90, mx in report:   # a gross-error check: float32 noise dominates the tails
        assert med <= 5e-2, (name, med, p90, mx)


def test_autograd_function_through_a_pose_loss(diff_world):
    import torch
    fw = _fw()
    sc, w, x0 = diff_world
    sc2, tp, tq = S.diff_peg_scene(n_envs=32, seed=2, n_substeps=sc.sim.n_substeps, n_iters=8)
    Rollout = fw.rollout_function()
    dev = torch.device("cuda")
    nb = len(x0[0])
    pegs = torch.arange(0, nb, 2, device=dev)
    ins = [torch.tensor(a, device=dev, requires_grad=True) for a in x0]
    mass = torch.tensor(np.where(np.arange(nb) % 2 == 0, sc.groups[0].bodies["mass"].reshape(-1), 0.0),
                        dtype=torch.float32, device=dev, requires_grad=True)
    mu = torch.tensor(sc.groups[0].bodies["mu"][:, 0], dtype=torch.float32, device=dev, requires_grad=True)
    pos, quat, lin, ang = Rollout.apply(w, sc.sim.n_substeps, sc.sim.n_iters, *ins, mass, mu)
    tpos = torch.tensor(tp, dtype=torch.float32, device=dev)
    tquat = torch.tensor(tq, dtype=torch.float32, device=dev)
    loss = ((pos[pegs] - tpos) ** 2).sum() + 1e-4 * ((quat[pegs] - tquat) ** 2).sum()
    loss.backward()
    # the same gradients straight from the ABI
    gp = torch.zeros(nb, 3, device=dev)
    gq = torch.zeros(nb, 4, device=dev)
    gp[pegs] = 2 * (pos[pegs] - tpos).detach()
    gq[pegs] = 2e-4 * (quat[pegs] - tquat).detach()
    z3 = torch.zeros(nb, 3, device=dev)
    ref = w.adjoint_rollout(gp, gq, z3, z3)
    for got, want in zip([ins[0].grad, ins[1].grad, ins[2].grad, ins[3].grad, mass.grad, mu.grad], ref):
        assert torch.allclose(got, want, rtol=1e-6, atol=1e-12)
    assert torch.isfinite(mass.grad).all() and mass.grad[pegs].abs().max() > 0
    assert mu.grad.abs().max() > 0


# ------------------------------------------------------------- config-3 size, untaped differences
def _env_tapes(t, n_envs):
    """per env, per substep: (contact records, row bits, clamp bit) of a tape"""
    S_, K = t["S"], t["K"]
    off, rec, rb, bb = t["c_off"], t["c_rec"], t["r_bits"], t["b_bits"]
    out = []
    for e in range(n_envs):
        parts = []
        for s in range(S_):
            a, b = off[s * n_envs + e], off[s * n_envs + e + 1]
            parts.append((rec[a:b].tobytes(), rb[K * a:K * b].tobytes(), int(bb[s * n_envs + e])))
        out.append(parts)
    return out


def test_config3_adjoint_against_untaped_central_differences():
    """The differentiable peg at its configured size (256 envs, one frame of 32 substeps x 8
    sweeps) against central differences of the FP64 oracle's own forward -- not a replay of
    a tape.  Each env is moved along its own random direction over all 14 inputs (position,
    rotation, linear and angular velocity, mass, friction; scaled by 1 mm, 0.01 rad, 1 cm/s,
    1 rad/s, the mass and 1) by +-h with h = 1e-6, and the oracle records its own decisions
    at x0 and at both ends.  Envs whose decisions (contacts with their SDF cells and branch
    bits, per-sweep clamp bits, |omega| clamp) are the same at all three points are kept:
    there the frame is one smooth function and its central difference is exact to O(h^2).
    On every kept env whose GPU tape also equals the oracle's, the GPU adjoint's
    directional derivative agrees to 1e-3 relative.  The kept and agreeing fractions are
    printed and floored.  (h = 1e-4 keeps no env of this workload: a jammed peg carries
    ~1,300 taped contacts and ~10,000 clamp bits per env, and a step of 0.1 um in position
    already moves some sample across an SDF cell or a reduction slot's winner.)"""
    fw = _fw()
    sc, tp, tq = S.diff_peg_scene(n_envs=256, seed=4)
    E, K, Sn = sc.n_envs, sc.sim.n_iters, sc.sim.n_substeps
    b0 = sc.groups[0].bodies
    x0 = [np.ascontiguousarray(b0[k].reshape(-1, b0[k].shape[-1]), np.float32) for k in ("pos", "quat", "linvel", "angvel")]
    nb = len(x0[0])
    pegs = np.arange(0, nb, 2)
    gw = fw.world_from_scene(sc)
    gw.set_state(*x0)
    gw.record_rollout(Sn, K)
    tg = _env_tapes(gw.get_tape(), E)
    rng = np.random.default_rng(11)
    g = [rng.normal(size=(nb, k)).astype(np.float32) for k in (3, 4, 3, 3)]
    g[0] *= 1e3
    for a in g:
        a[1::2] = 0.0
    adj = gw.adjoint_rollout(*g)
    ow = O.world_from_scene(sc, lazy_bake=True)
    mass0 = np.array([ow.body_mass(int(b)) for b in pegs])
    mu0 = np.array([ow.pair_mu(e) for e in range(E)])
    x64 = [a.astype(np.float64) for a in x0]

    def record(xs, mass, mu):
        ow.set_state(*xs)
        for e, b in enumerate(pegs):
            ow.set_body_mass(int(b), float(mass[e]))
        for e in range(E):
            ow.set_pair_mu(e, float(mu[e]))
        ow.diff_record(Sn, K)
        return _env_tapes(ow.get_tape(), E), [a.copy() for a in ow.state()]

    h = 1e-6
    scale = dict(pos=1e-3, rot=1e-2, lin=1e-2, ang=1.0)
    d = {k: rng.normal(size=(E, 3)) for k in scale}
    dm, dmu = rng.normal(size=E), rng.normal(size=E)

    def perturbed(sign):
        xs = [a.copy() for a in x64]
        for e, bdy in enumerate(pegs):
            xs[0][bdy] += sign * h * scale["pos"] * d["pos"][e]
            xs[2][bdy] += sign * h * scale["lin"] * d["lin"][e]
            xs[3][bdy] += sign * h * scale["ang"] * d["ang"][e]
            th = sign * h * scale["rot"] * d["rot"][e]
            xs[1][bdy] = S.quat_mul(S.quat_axis_angle(th / np.linalg.norm(th), np.linalg.norm(th)), x64[1][bdy])
        return xs, mass0 * (1.0 + sign * h * dm), mu0 + sign * h * dmu

    to, _ = record(x64, mass0, mu0)
    tpl, xp = record(*perturbed(+1.0))
    tmi, xm = record(*perturbed(-1.0))
    kept = np.array([to[e] == tpl[e] == tmi[e] for e in range(E)])
    agree = np.array([tg[e] == to[e] for e in range(E)])
    g64 = [a.astype(np.float64) for a in g]
    loss = lambda X: sum((gi * xi).sum(axis=1) for gi, xi in zip(g64, X))[pegs]
    fd = (loss(xp) - loss(xm)) / 2.0
    an = np.zeros(E)
    for e, bdy in enumerate(pegs):
        an[e] += adj[0][bdy] @ (h * scale["pos"] * d["pos"][e]) + adj[2][bdy] @ (h * scale["lin"] * d["lin"][e])
        an[e] += adj[3][bdy] @ (h * scale["ang"] * d["ang"][e])
        th = h * scale["rot"] * d["rot"][e]
        an[e] += adj[1][bdy].astype(np.float64) @ (0.5 * S.quat_mul(np.array([th[0], th[1], th[2], 0.0]), x64[1][bdy]))
        an[e] += adj[4][bdy] * mass0[e] * h * dm[e] + adj[5][e] * h * dmu[e]
    err = np.abs(an - fd) / np.maximum(np.abs(fd), 1e-2 * np.abs(fd).max())
    both = kept & agree
    print(f"\nconfig-3 adjoint: {kept.sum()} of {E} envs keep every decision within +-h, the GPU tape equals the "
          f"oracle's in {agree.sum()}, both in {both.sum()}; GPU directional derivative vs untaped FP64 central "
          f"differences there: median {np.median(err[both]):.1e}, max {err[both].max():.1e}; "
          f"over the other envs median {np.median(err[~both]):.1e}")
    assert kept.sum() >= 0.5 * E and both.sum() >= 0.3 * E, (kept.sum(), both.sum())
    assert np.all(err[both] <= 1e-3), float(err[both].max())
