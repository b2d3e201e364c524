"""Pile envs on the GPU (R20): one env of many nuts over a plate whose pairs the pair-list
kernel finds again at every detection (bounding spheres within the contact offset plus
two voxels, (i, j) order), detected by the same narrow phase and Algorithm 1 as listed
pairs, and solved colour by colour by one block per pile -- against the FP64 oracle.

Tolerances as for the listed-pair scenes: the pair list identical (a pair whose sphere
test is within 1e-6 of its limit may go either way); contact sets per pair identical
where the pair's decisions have margin and in bulk otherwise; identical contacts solved
for one substep to 1e-6 m / rad, with identical colours; a frame to 2e-4 m / 2e-3 rad.
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


def _same_pairs(sc, gw, pos, gab, oab):
    """the two pair lists hold the same pairs, except pairs right at the sphere limit
    (radius_a + radius_b + offset + 2 h_b, the SDF body's voxel h_b)"""
    g, o = {tuple(p) for p in gab}, {tuple(p) for p in oab}
    b = sc.piles[0]
    r = [float(max(np.linalg.norm(a.verts, axis=1).max(),
                   0 if a.samples is None else np.linalg.norm(a.samples, axis=1).max())) for a in sc.assets]
    for (i, j) in g ^ o:   # (sample body, SDF body)
        hj = float(gw.get_sdf(int(b["asset"][j]), values=False)[1])
        d = float(np.linalg.norm(pos[i].astype(np.float64) - pos[j].astype(np.float64)))
        lim = r[b["asset"][i]] + r[b["asset"][j]] + 1e-4 + 2 * hj
        assert abs(d - lim) <= 1e-6 * lim, ((i, j), d, lim)
    return len(g ^ o)


@pytest.fixture(scope="module")
def heap64():
    fw = _fw()
    sc = S.nut_pile_env_scene(64, seed=1, mode="heap")
    gw = fw.world_from_scene(sc)
    ow = O.world_from_scene(sc, lazy_bake=True, margin_len=MARGIN_LEN, margin_dot=MARGIN_DOT)
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    gw.collide()
    ow.reset_margins()
    ow.collide()
    return sc, gw, ow


def test_env_info_and_launch_count(heap64):
    sc, gw, ow = heap64
    fb, nb, fp, np_ = gw.env_info(0)
    assert (fb, nb, fp, np_) == (0, 65, -1, -1)
    assert gw.counts() == (1, 65, 0)
    # per substep: pair list, maps, query, reduction, the pile solve's prep and sweeps
    assert gw.launches_per_step(4) == 24


def test_pair_list_matches_oracle(heap64):
    sc, gw, ow = heap64
    gab, _ = gw.pile_pairs(0)
    oab, _ = ow.pile_pairs(0)
    pos = gw.get_state()[0]
    n_diff = _same_pairs(sc, gw, pos, gab, oab)
    assert len(gab) > 150, len(gab)
    if n_diff == 0:
        np.testing.assert_array_equal(gab, oab)   # the same pairs in the same order


def test_contacts_per_pair_where_decisions_have_margin(heap64):
    sc, gw, ow = heap64
    gab, _ = gw.pile_pairs(0)
    gc_all = gw.get_contacts(0)
    compared = bulk = with_contacts = 0
    for k in range(len(gab)):
        gc = gc_all[gc_all["pair"] == k]
        oc = ow.pair_contacts(0, k)
        with_contacts += len(oc) > 0
        ml, md = ow.pair_margins(0, k)
        if ml >= MARGIN_LEN and md >= MARGIN_DOT:
            assert list(gc["sample"]) == list(oc["sample"]), k
            assert list(gc["patch"]) == list(oc["patch"]), k
            h = float(gw.get_sdf(int(sc.piles[0]["asset"][gab[k][1]]), values=False)[1])
            assert np.all(np.abs(gc["phi"] - oc["phi"]) <= 5e-5 * h)
            compared += len(oc) > 0
        else:
            bulk += 1
            if len(oc) == 0:
                assert len(gc) == 0
                continue
            common = len(set(gc["sample"]) & set(oc["sample"]))
            assert common >= 0.8 * max(len(gc), len(oc)), (k, common, len(gc), len(oc))
            assert abs(len(gc) - len(oc)) <= max(3, 0.15 * len(oc)), (k, len(gc), len(oc))
    print(f"pairs {len(gab)}, with contacts {with_contacts}, compared exactly {compared}, in bulk {bulk}")
    # flat faces resting on flat faces tie many of Algorithm 1's decisions (15 of the 81
    # pairs with contacts have every margin above the thresholds for this seed)
    assert with_contacts >= 60 and compared >= 12, (with_contacts, compared)


def test_solve_identical_contacts_one_substep_and_colours(heap64):
    """The oracle's contacts (rounded to float32 on both sides) into both worlds, one
    substep without detection: the same colours, and the state to 1e-6 m / rad."""
    sc, gw, ow = heap64
    fw = _fw()
    hs = sc.sim.dt / sc.sim.n_substeps
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    ow.collide()
    oab, _ = ow.pile_pairs(0)
    gab, _ = gw.pile_pairs(0)
    np.testing.assert_array_equal(gab, oab)
    parts = []
    for k in range(len(oab)):
        oc = ow.pair_contacts(0, k)
        gc = np.zeros(len(oc), fw.CONTACT_DTYPE)
        gc["sample"], gc["patch"], gc["phi"] = oc["sample"], oc["patch"], oc["phi"]
        gc["xa"], gc["n"] = oc["xa"], oc["n"]
        gc["xb"] = gc["xa"] - gc["phi"][:, None] * gc["n"]
        gc["pair"] = k
        same = oc.copy()
        same["phi"] = gc["phi"]
        same["xa"], same["n"] = gc["xa"], gc["n"]
        same["xb"] = same["xa"] - same["phi"][:, None] * same["n"]
        ow.set_pair_contacts(0, k, same)
        parts.append(gc)
    gw.set_contacts(0, np.concatenate(parts))
    gw.substep(hs, sc.sim.n_iters, detect=False)
    ow.substep(hs, sc.sim.n_iters, detect=False)
    _, gcol = gw.pile_pairs(0)
    _, ocol = ow.pile_pairs(0)
    np.testing.assert_array_equal(gcol, ocol)
    assert gcol.max() >= 2
    gp, gq, gv, gwv = gw.get_state()
    op, oq, ov, owv = ow.state()
    assert np.abs(gp - op).max() <= 1e-6
    assert max(_rot_angle(gq[i].astype(np.float64), oq[i]) for i in range(len(gq))) <= 1e-6
    assert np.abs(gv - ov).max() <= 1e-4 * max(1.0, float(np.abs(ov).max()))


def test_one_frame_of_the_heap(heap64):
    sc, gw, ow = heap64
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    gw.step(sc.sim.n_substeps, sc.sim.n_iters)
    ow.step(sc.sim.n_substeps, sc.sim.n_iters)
    gp, gq, _, _ = gw.get_state()
    op, oq, _, _ = ow.state()
    assert np.abs(gp - op).max() <= 2e-4
    assert max(_rot_angle(gq[i].astype(np.float64), oq[i]) for i in range(len(gq))) <= 2e-3


def test_pair_capacity_overflow_is_reported():
    fw = _fw()
    sc = S.nut_pile_env_scene(16, seed=3, mode="heap", n_samples=2000, sdf_res=64, plate_sdf_res=64)
    w = fw.World(fw.default_config())
    for a in sc.assets:
        i = w.add_mesh_asset(a.verts, a.tris, a.samples, a.density)
        w.bake_sdf(i, a.sdf_res, a.sdf_pad, True)
    env = w.add_pile(sc.piles[0], max_pairs=5)
    w.collide()
    with pytest.raises(fw.FwError) as e:
        w.sync()
    assert "than fit" in str(e.value)
    ab, _ = w.pile_pairs(env)
    assert len(ab) == 5
    w.close()


def test_full_size_drop_pile_1023_nuts():
    """The bench workload (1023 nuts dropped from a lattice over the plate, one pile env):
    its pair list at the initial poses equals the oracle's broad phase, a few frames run
    without a non-finite state or an overflow, and the sampled pairs' contacts after
    them match the oracle's detection of those pairs at the same poses."""
    fw = _fw()
    sc = S.nut_pile_env_scene(1023, seed=0, mode="drop")
    gw = fw.world_from_scene(sc, max_patches=128)
    ow = O.world_from_scene(sc, lazy_bake=True, margin_len=MARGIN_LEN, margin_dot=MARGIN_DOT)
    gw.collide()
    gab, _ = gw.pile_pairs(0)
    oab, _ = ow.find_pile_pairs(0)
    pos = gw.get_state()[0]
    assert _same_pairs(sc, gw, pos, gab, oab) <= 2
    assert len(gab) >= 1023          # every nut over the plate
    for _ in range(30):
        gw.step(sc.sim.n_substeps, sc.sim.n_iters)
    gw.sync()
    p, q, v, w = gw.get_state()
    assert np.all(np.isfinite(p)) and np.all(np.isfinite(v))
    assert p[:-1, 2].min() > -0.002                 # nothing fell through the plate
    gw.collide()
    gab, _ = gw.pile_pairs(0)
    gc_all = gw.get_contacts(0)
    # the oracle detects a sample of the GPU's pairs as listed pairs at the same poses
    rng = np.random.default_rng(0)
    counts = np.bincount(gc_all["pair"], minlength=len(gab))
    pick = rng.choice(np.nonzero(counts)[0], size=min(12, int((counts > 0).sum())), replace=False)
    import dataclasses
    b = sc.piles[0].copy()
    b["pos"], b["quat"], b["linvel"], b["angvel"] = p, q, v, w
    lw = O.world_from_scene(dataclasses.replace(sc, piles=[], groups=[S.EnvGroup(b[None, :], gab[pick])]),
                            lazy_bake=True, margin_len=MARGIN_LEN, margin_dot=MARGIN_DOT)
    lw.set_state(p, q, v, w)
    lw.collide()
    exact = 0
    for m, k in enumerate(pick):
        gc = gc_all[gc_all["pair"] == k]
        oc = lw.pair_contacts(0, m)
        ml, md = lw.pair_margins(0, m)
        if ml >= MARGIN_LEN and md >= MARGIN_DOT:
            assert list(gc["sample"]) == list(oc["sample"])
            exact += 1
        else:
            common = len(set(gc["sample"]) & set(oc["sample"]))
            assert common >= 0.8 * max(len(gc), len(oc), 1)
    print(f"pairs {len(gab)}, with contacts {(counts > 0).sum()}, contacts {len(gc_all)}, sampled exact {exact}")
    gw.close()


@pytest.mark.parametrize("kind, sdf_res", [("torus", 64), ("bowl", 128)])
def test_torus_and_bowl_heaps_match_oracle(kind, sdf_res):
    """The paper's other two pile bodies (Sec. III-D: piles of 1,024 toruses and of 1,024
    bowls in one env), 16 of them in stacks over a plate -- toruses lying flat on each other,
    bowls nested in each other -- through the same pile path: the pair list identical,
    contacts per pair identical where the pair's margins allow (most pairs: the surfaces are
    smooth), one substep on identical contacts with identical colours to 1e-6."""
    fw = _fw()
    sc = S.pile_env_scene(kind, 16, seed=3, mode="heap", n_samples=3000, sdf_res=sdf_res, plate_sdf_res=64)
    gw = fw.world_from_scene(sc)
    ow = O.world_from_scene(sc, lazy_bake=True, margin_len=MARGIN_LEN, margin_dot=MARGIN_DOT)
    p, q, v, w = gw.get_state()
    ow.set_state(p, q, v, w)
    gw.collide()
    ow.reset_margins()
    ow.collide()
    gab, _ = gw.pile_pairs(0)
    oab, _ = ow.pile_pairs(0)
    assert _same_pairs(sc, gw, p, gab, oab) == 0
    np.testing.assert_array_equal(gab, oab)
    gc_all = gw.get_contacts(0)
    exact = with_contacts = 0
    parts = []
    for k in range(len(oab)):
        gc = gc_all[gc_all["pair"] == k]
        oc = ow.pair_contacts(0, k)
        with_contacts += len(oc) > 0
        ml, md = ow.pair_margins(0, k)
        if ml >= MARGIN_LEN and md >= MARGIN_DOT:
            assert list(gc["sample"]) == list(oc["sample"]), k
            assert list(gc["patch"]) == list(oc["patch"]), k
            exact += len(oc) > 0
        else:
            common = len(set(gc["sample"]) & set(oc["sample"]))
            assert common >= 0.8 * max(len(gc), len(oc), 1), (k, common, len(gc), len(oc))
        g = np.zeros(len(oc), fw.CONTACT_DTYPE)
        g["sample"], g["patch"], g["phi"] = oc["sample"], oc["patch"], oc["phi"]
        g["xa"], g["n"] = oc["xa"], oc["n"]
        g["xb"] = g["xa"] - g["phi"][:, None] * g["n"]
        g["pair"] = k
        same = oc.copy()
        same["phi"], same["xa"], same["n"] = g["phi"], g["xa"], g["n"]
        same["xb"] = same["xa"] - same["phi"][:, None] * same["n"]
        ow.set_pair_contacts(0, k, same)
        parts.append(g)
    print(f"{kind} heap: pairs {len(oab)}, with contacts {with_contacts}, compared exactly {exact}")
    assert with_contacts >= 15 and exact >= with_contacts // 2, (with_contacts, exact)
    gw.set_contacts(0, np.concatenate(parts))
    hs = sc.sim.dt / sc.sim.n_substeps
    gw.substep(hs, sc.sim.n_iters, detect=False)
    ow.substep(hs, sc.sim.n_iters, detect=False)
    np.testing.assert_array_equal(gw.pile_pairs(0)[1], ow.pile_pairs(0)[1])
    gp, gq, gv, _ = gw.get_state()
    op, oq, ov, _ = ow.state()
    assert np.abs(gp - op).max() <= 1e-6
    assert max(_rot_angle(gq[i].astype(np.float64), oq[i]) for i in range(len(gq))) <= 1e-6
    assert np.abs(gv - ov).max() <= 1e-4 * max(1.0, float(np.abs(ov).max()))
    gw.close()
