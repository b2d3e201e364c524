"""Failure detection through the ABI, made on the host (no test faults, traps or hangs a
GPU): a non-finite state injected into the inputs surfaces as FW_ERR_NONFINITE from the
device status word at the next synchronising call; bad arguments and out-of-order calls
are refused with FW_ERR_ARG / FW_ERR_STATE before anything is enqueued; an output buffer
too small is FW_ERR_OVERFLOW with the needed size; after any of them the world still
steps and agrees with an untouched world."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from paper_2205_03532_b300 import scenes as S

ERR_ARG, ERR_STATE, ERR_NONFINITE, ERR_OVERFLOW = -1, -4, -5, -6


def _fw():
    from paper_2205_03532_b300 import fw
    return fw


def _peg(n_envs=4):
    sc = S.peg_in_hole_scene(n_envs=n_envs, seed=2)
    sc.groups[0].bodies["pos"][:, 0, 2] = 12.5e-3 - 2e-3
    return sc


def _status(e):
    return e.value.status


def test_nan_state_is_reported_and_the_world_recovers():
    fw = _fw()
    sc = _peg()
    w, ref = fw.world_from_scene(sc), fw.world_from_scene(sc)
    p, q, v, om = w.get_state()
    bad = v.copy()
    bad[2, 1] = np.nan
    w.set_state(p, q, bad, om)
    w.step(4, 16)
    with pytest.raises(fw.FwError) as e:
        w.get_state()
    assert _status(e) == ERR_NONFINITE
    # the status word is cleared once reported; a clean state steps as an untouched world
    w.set_state(p, q, v, om)
    ref.set_state(p, q, v, om)
    w.step(4, 16)
    ref.step(4, 16)
    for x, y in zip(w.get_state(), ref.get_state()):
        np.testing.assert_array_equal(x, y)
    w.close()
    ref.close()


def test_bad_arguments_are_refused():
    fw = _fw()
    for k, v in (("batch_size", 512), ("patch_dirs", 5), ("max_patches", 0), ("dt", 0.0), ("contact_gen", 2),
                 ("sdf_band", -1.0), ("solver", 3)):
        with pytest.raises(fw.FwError) as e:
            fw.World(**{k: v})
        assert _status(e) == ERR_ARG, k
    w = fw.World()
    V, T = S.box_mesh(0.01, 0.01, 0.01)
    with pytest.raises(fw.FwError) as e:
        w.add_mesh_asset(V, np.array([[0, 1, 99]], np.int32), None)       # vertex index out of range
    assert _status(e) == ERR_ARG
    a = w.add_mesh_asset(V, T, S.sample_surface(V, T, 100, np.random.default_rng(0)))
    b = w.add_mesh_asset(V, T, None)
    with pytest.raises(fw.FwError) as e:
        w.bake_sdf(b, 1, 1e-3)                                           # resolution below 2
    assert _status(e) == ERR_ARG
    bodies = np.zeros((1, 2), S.BODY_DTYPE)
    bodies[0, 0] = S._body(a, S.DYNAMIC, (0, 0, 0.03), (0, 0, 0, 1), 0.5)
    bodies[0, 1] = S._body(b, S.STATIC, (0, 0, 0), (0, 0, 0, 1), 0.5)
    with pytest.raises(fw.FwError) as e:
        w.add_env_bodies(bodies, np.array([[0, 1]], np.int32))          # SDF body without an SDF yet
    assert _status(e) == ERR_STATE
    w.bake_sdf(b, 32, 2e-3)
    with pytest.raises(fw.FwError) as e:
        w.add_env_bodies(bodies, np.array([[0, 0]], np.int32))          # a body paired with itself
    assert _status(e) == ERR_ARG
    w.add_env_bodies(bodies, np.array([[0, 1]], np.int32))
    with pytest.raises(fw.FwError) as e:
        w.step(0, 16)
    assert _status(e) == ERR_ARG
    with pytest.raises(fw.FwError) as e:
        w.query_sdf(a, np.zeros((4, 3), np.float32))                   # the point body has no SDF
    assert _status(e) == ERR_STATE
    w.step(4, 16)                                                      # still usable
    assert np.all(np.isfinite(w.get_state()[0]))
    w.close()


def test_contact_buffer_too_small_reports_the_size():
    fw = _fw()
    sc = _peg(n_envs=2)
    w = fw.world_from_scene(sc)
    w.collide()
    n_all = len(w.get_contacts(0))
    assert n_all > 2
    out = np.zeros(2, fw.CONTACT_DTYPE)
    n = C.c_int()
    st = w.lib.fw_get_contacts(w.h, 0, out.ctypes.data, 2, C.byref(n))
    assert st == ERR_OVERFLOW and n.value == n_all
    w.close()


def test_rollout_recording_refuses_per_triangle_contacts():
    """The adjoint's tape rebuilds each contact from its surface sample; a per-triangle
    contact (contact_gen = 1) has none, so recording is refused on the host before anything
    is enqueued.  Only the refusal is exercised: no kernel runs with such a world."""
    fw = _fw()
    sc = _peg(n_envs=2)
    w = fw.world_from_scene(sc, contact_gen=1)
    for call in (lambda: w.record_rollout(4, 8), lambda: w.step_fwd_ckpt(4, 8)):
        with pytest.raises(fw.FwError) as e:
            call()
        assert _status(e) == ERR_ARG and "contact_gen" in str(e.value)
    with pytest.raises(fw.FwError) as e:
        w.replay_rollout()                                             # nothing was recorded
    assert _status(e) == ERR_STATE
    w.close()


def test_env_info_locates_bodies_of_uneven_env_groups():
    """Envs added by several calls with different structures: fw_get_env_info gives each
    env's first body and pair in the global order of fw_get_state and the pair adjoints."""
    fw = _fw()
    w = fw.World()
    V, T = S.box_mesh(0.01, 0.01, 0.01)
    a = w.add_mesh_asset(V, T, S.sample_surface(V, T, 100, np.random.default_rng(0)))
    b = w.add_mesh_asset(V, T, None)
    w.bake_sdf(b, 32, 2e-3)
    one = np.zeros((3, 1), S.BODY_DTYPE)
    for e in range(3):
        one[e, 0] = S._body(a, S.DYNAMIC, (0.1 * e, 0, 0.5), (0, 0, 0, 1), 0.5)
    two = np.zeros((2, 2), S.BODY_DTYPE)
    for e in range(2):
        two[e, 0] = S._body(a, S.DYNAMIC, (0, 0.1 * e, 0.03), (0, 0, 0, 1), 0.5)
        two[e, 1] = S._body(b, S.STATIC, (0, 0.1 * e, 0), (0, 0, 0, 1), 0.5)
    assert w.add_env_bodies(one, np.zeros((0, 2), np.int32)) == 0
    assert w.add_env_bodies(two, np.array([[0, 1]], np.int32)) == 3
    assert [w.env_info(e) for e in range(5)] == [(0, 1, 0, 0), (1, 1, 0, 0), (2, 1, 0, 0), (3, 2, 0, 1), (5, 2, 1, 1)]
    p = w.get_state()[0]
    np.testing.assert_array_equal(p[5], two[1, 0]["pos"])
    with pytest.raises(fw.FwError) as e:
        w.env_info(5)
    assert _status(e) == ERR_ARG
    w.close()


def test_a_solve_chunk_wait_that_runs_out_is_reported_and_the_world_recovers():
    """Failure detection on the device without a fault: with the test hook, the solve's row
    stream issues no chunk copy, so its first bounded mbarrier wait sees no arrival and gives
    up (after 2^20 polls, tens of milliseconds).  The kernel ends, the next synchronising call reports
    FW_ERR_TIMEOUT, and once the hook is off the same world steps on as a fresh one does."""
    import time
    fw = _fw()
    sc = S.nut_bolt_scene(n_envs=4, seed=2)
    w = fw.world_from_scene(sc)
    ref = fw.world_from_scene(sc)
    s0 = [a.copy() for a in w.get_state()]
    w.test_stall(2)
    t0 = time.time()
    w.step(1, 8)
    with pytest.raises(fw.FwError) as e:
        w.sync()
    assert _status(e) == -7 and "wait" in str(e.value)
    assert time.time() - t0 < 30
    w.test_stall(0)
    w.set_state(*s0)       # (set_state normalises the quaternions: the reference takes it too)
    ref.set_state(*s0)
    w.step(1, 8)
    ref.step(1, 8)
    for a, b in zip(w.get_state(), ref.get_state()):
        np.testing.assert_array_equal(a, b)
    w.close()
    ref.close()


def test_a_pile_grid_barrier_that_runs_out_is_reported_and_the_world_recovers():
    """The pile sweep kernel's grid barrier with the test hook waits for one block more than
    the cooperative launch has: every block gives up after about a second, stops waiting at
    the later barriers, and the launch ends; FW_ERR_TIMEOUT is reported and the world steps
    on afterwards."""
    import time
    fw = _fw()
    sc = S.nut_pile_env_scene(12, seed=3, mode="heap", n_samples=2000, sdf_res=64, plate_sdf_res=64)
    w = fw.world_from_scene(sc)
    ref = fw.world_from_scene(sc)
    s0 = [a.copy() for a in w.get_state()]
    w.test_stall(1)
    t0 = time.time()
    w.step(1, 4)
    with pytest.raises(fw.FwError) as e:
        w.sync()
    assert _status(e) == -7
    assert time.time() - t0 < 30
    w.test_stall(0)
    w.set_state(*s0)
    ref.set_state(*s0)
    w.step(1, 4)
    ref.step(1, 4)
    for a, b in zip(w.get_state(), ref.get_state()):
        np.testing.assert_array_equal(a, b)
    w.close()
    ref.close()
