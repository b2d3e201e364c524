"""The narrow phase's cull of sample groups (fw_set_query_cull; Sec. III-A): a group of 32
consecutive samples is skipped only when none of them can be a candidate, so the
candidates, the contacts and the states after them are the same bit for bit with the cull
on and off -- on the peg, the nut-bolt pair, the mixed nut-bolt sizes, the gear train
(FP16 SDFs), the 7-nut piles (bodies apart, coming together) and the pile envs (nuts,
toruses and bowls heaped on a plate; pair lists found on the device).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from paper_2205_03532_b300 import scenes as S

SCENES = {
    "peg": lambda: (S.peg_in_hole_scene(n_envs=4, seed=2), False),
    "nut": lambda: (S.nut_bolt_scene(n_envs=6, seed=1), False),
    "mixed": lambda: (S.mixed_nut_bolt_scene(n_envs=8, seed=3), True),
    "gears": lambda: (S.gear_scene(n_envs=6, seed=4), True),
    "pile": lambda: (S.pile_scene(n_envs=3, seed=5, n_nuts=7), False),
    "pile_env_nut": lambda: (S.nut_pile_env_scene(64, seed=1, mode="heap"), False),
    "pile_env_torus": lambda: (S.pile_env_scene("torus", 16, seed=3, mode="heap", n_samples=3000, sdf_res=64,
                                                plate_sdf_res=64), False),
    "pile_env_bowl": lambda: (S.pile_env_scene("bowl", 16, seed=3, mode="heap", n_samples=3000, sdf_res=128,
                                               plate_sdf_res=64), False),
}


@pytest.mark.parametrize("name", sorted(SCENES))
def test_cull_changes_nothing(name):
    from paper_2205_03532_b300 import fw
    sc, fp16 = SCENES[name]()
    runs = []
    for on in (True, False):
        w = fw.world_from_scene(sc, fp16=fp16)
        w.set_query_cull(on)
        n_env = w.counts()[0]
        stats = []
        for _ in range(3):
            w.step(sc.sim.n_substeps, sc.sim.n_iters)
            stats.append(w.detect_stats())
        runs.append((w.get_state(), [w.get_contacts(e) for e in range(n_env)], stats))
        w.close()
    (s_on, c_on, d_on), (s_off, c_off, d_off) = runs
    assert d_on == d_off
    assert sum(len(c) for c in c_on) > 0, name          # the scene is in contact
    for a, b in zip(c_on, c_off):
        assert a.tobytes() == b.tobytes()
    for a, b in zip(s_on, s_off):
        np.testing.assert_array_equal(a, b)


def test_cull_switch_refuses_other_values():
    from paper_2205_03532_b300 import fw
    w = fw.world_from_scene(S.peg_in_hole_scene(n_envs=1, seed=0))
    with pytest.raises(fw.FwError):
        w._check(w.lib.fw_set_query_cull(w.h, 2))
    w.close()


def test_cull_setting_reads_back_and_the_autotuner_changes_no_contact():
    """fw_get_query_cull reports the setting in use (on by default); the detection
    autotuner may turn it either way, and the contacts it leaves are those of the setting
    before it"""
    from paper_2205_03532_b300 import fw
    sc = S.nut_bolt_scene(n_envs=8, seed=2)
    w = fw.world_from_scene(sc)
    assert w.query_cull() is True
    w.set_query_cull(False)
    assert w.query_cull() is False
    w.set_query_cull(True)
    w.step(sc.sim.n_substeps, sc.sim.n_iters)
    w.collide()
    before = [w.get_contacts(e).tobytes() for e in range(w.counts()[0])]
    w.autotune_detect(trials=2)
    assert isinstance(w.query_cull(), bool)
    after = [w.get_contacts(e).tobytes() for e in range(w.counts()[0])]
    assert before == after
    w.set_query_cull(not w.query_cull())
    w.collide()
    assert [w.get_contacts(e).tobytes() for e in range(w.counts()[0])] == before
    w.close()
