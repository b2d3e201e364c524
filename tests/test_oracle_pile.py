"""Piles of nuts through the oracle (several free bodies per env, coupled through
nut-plate and nut-nut contacts; the general Gauss-Seidel form over all the env's pairs),
pinned by statics rather than by the oracle's own code: stacks of nuts lying flat on a
plate, each sunk 0.02 mm into its support, are in equilibrium -- after a third of a
second no nut has moved by more than a fraction of a millimetre or kept any speed, and
pairs whose nuts are apart have no contacts."""
import numpy as np

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


def test_stacks_of_nuts_stay_at_rest():
    sc = S.pile_scene(n_envs=2, seed=1, n_nuts=4, mode="stacks")
    w = O.world_from_scene(sc, lazy_bake=True)
    w.collide()
    pairs = sc.groups[0].pairs
    b = sc.groups[0].bodies
    r = float(np.linalg.norm(sc.assets[0].verts, axis=1).max())
    for env in range(sc.n_envs):
        n = [len(w.pair_contacts(env, k)) for k in range(len(pairs))]
        for k, (i, j) in enumerate(pairs):
            if j < 4 and np.linalg.norm(b["pos"][env, i] - b["pos"][env, j]) > 2 * r + 1e-3:
                assert n[k] == 0, (env, k)
        assert sum(n) > 20
    p0 = w.state()[0].copy()
    for _ in range(20):
        w.step(sc.sim.n_substeps, sc.sim.n_iters)
    p, q, v, om = w.state()
    nuts = [i for i in range(len(p)) if i % 5 != 4]
    assert np.abs(p[nuts] - p0[nuts]).max() <= 2e-4
    assert np.abs(v[nuts]).max() <= 2e-3 and np.abs(om[nuts]).max() <= 5e-2
    assert np.all(p[nuts, 2] > 0.0)                     # every nut above the plate's top face


# ----------------------------------------------------------------------------------------
# pile envs (R20): one env whose pairs a broad phase finds at every detection
# ----------------------------------------------------------------------------------------
import dataclasses

import pytest


def _small_heap(n_nuts=9, seed=2, **kw):
    return S.nut_pile_env_scene(n_nuts, seed=seed, mode="heap", n_samples=2000, sdf_res=64, plate_sdf_res=64,
                                **kw)


def _listed(sc, pairs):
    """the pile's bodies as one env of listed pairs (the path pinned by the other tests)"""
    b = sc.piles[0][None, :]
    return dataclasses.replace(sc, groups=[S.EnvGroup(b, np.asarray(pairs, np.int32).reshape(-1, 2))], piles=[])


def _rule_pairs(sc, w):
    """every (sample body, SDF body) pair the rule allows for bodies i < j, at least one
    movable, ignoring distance"""
    b = sc.piles[0]
    has_s = [sc.assets[k].samples is not None for k in range(len(sc.assets))]
    has_g = [sc.assets[k].sdf_res is not None for k in range(len(sc.assets))]
    out = []
    for i in range(len(b)):
        for j in range(i + 1, len(b)):
            if b["type"][i] != S.DYNAMIC and b["type"][j] != S.DYNAMIC:
                continue
            ai, aj = b["asset"][i], b["asset"][j]
            if has_s[ai] and has_g[aj]:
                out.append((i, j))
            elif has_s[aj] and has_g[ai]:
                out.append((j, i))
    return out


@pytest.fixture(scope="module")
def heap9():
    sc = _small_heap()
    w = O.world_from_scene(sc, lazy_bake=True)
    w.collide()
    return sc, w


def test_pile_broad_phase_drops_no_contact(heap9):
    """Brute force: every pair the rule allows, detected as a listed pair.  The pile's list
    holds exactly the allowed pairs within reach, in (i, j) order; each has the contacts of
    its listed twin, and every allowed pair left out has none."""
    sc, w = heap9
    ab, _ = w.pile_pairs(0)
    everything = _rule_pairs(sc, w)
    wl = O.world_from_scene(_listed(sc, everything), lazy_bake=True)
    wl.collide()
    listed = {p: k for k, p in enumerate(everything)}
    kept = [tuple(p) for p in ab]
    assert kept == sorted(kept, key=lambda p: (min(p), max(p)))      # (i, j) order
    assert set(kept) <= set(everything)
    n_dropped_checked = 0
    for p, k in listed.items():
        c = wl.pair_contacts(0, k)
        if p in kept:
            g = w.pair_contacts(0, kept.index(p))
            assert len(g) == len(c)
            for f in ("sample", "patch", "phi", "xa", "n"):
                np.testing.assert_array_equal(g[f], c[f])
        else:
            assert len(c) == 0, p
            n_dropped_checked += 1
    assert n_dropped_checked > 10 and sum(len(w.pair_contacts(0, k)) for k in range(len(kept))) > 50


def test_pile_solve_is_the_listed_solve_in_colour_order(heap9):
    """One substep of the pile equals, to the last bit, the substep of the same bodies with
    the same contacts as listed pairs given in the pile's colour order (colour by colour,
    pair order within a colour): the pile solve is a Gauss-Seidel sweep in that order."""
    sc, w = heap9
    hs = sc.sim.dt / sc.sim.n_substeps
    w.substep(hs, sc.sim.n_iters, detect=False)
    ab, col = w.pile_pairs(0)
    assert (col >= 0).sum() > 5 and col.max() >= 1
    order = sorted(range(len(ab)), key=lambda k: (col[k] if col[k] >= 0 else 10 ** 6, k))
    wl = O.world_from_scene(_listed(sc, ab[order]), lazy_bake=True)   # the same initial state
    wl.collide()
    wl.substep(hs, sc.sim.n_iters, detect=False)
    for a, b in zip(w.state(), wl.state()):
        np.testing.assert_array_equal(a, b)
    # and in plain pair order the sweep is a different one (the order matters)
    wp = O.world_from_scene(_listed(sc, ab), lazy_bake=True)
    wp.collide()
    wp.substep(hs, sc.sim.n_iters, detect=False)
    assert not np.array_equal(w.state()[2], wp.state()[2])


def test_pile_colours_separate_pairs_that_share_a_movable_body(heap9):
    sc, w = heap9
    ab, col = w.pile_pairs(0)
    movable = sc.piles[0]["type"] == S.DYNAMIC
    n = np.array([len(w.pair_contacts(0, k)) for k in range(len(ab))])
    assert np.all((col >= 0) == (n > 0))
    assert set(col[col >= 0]) == set(range(col.max() + 1))            # colours 0.. without gaps
    for k in range(len(ab)):
        for m in range(k + 1, len(ab)):
            if col[k] < 0 or col[k] != col[m] or col[k] == 63:
                continue
            shared = set(ab[k]) & set(ab[m])
            assert not any(movable[i] for i in shared), (k, m, ab[k], ab[m])


def test_pile_frictionless_collision_conserves_momentum():
    """No gravity, no friction, no plate: three nuts of a stack sunk into each other and a
    fourth pressed against them, thrown at each other.  Every contact impulse acts on its
    two bodies with opposite signs, so the total linear momentum stays what it was."""
    sc = _small_heap(n_nuts=12, seed=4, mu=0.0)
    b = sc.piles[0]
    keep = [k for k in range(len(b) - 1)][:6]                      # nuts only
    nb = b[keep].copy()
    rng = np.random.default_rng(5)
    nb["linvel"] = rng.uniform(-0.05, 0.05, (len(nb), 3))
    nb["angvel"] = rng.uniform(-1.0, 1.0, (len(nb), 3))
    sc2 = dataclasses.replace(sc, piles=[nb])
    w = O.world_from_scene(sc2, lazy_bake=True, gravity=(0.0, 0.0, 0.0))
    m = np.array([w.mass(0)[0]] * len(nb))
    p0 = (m[:, None] * w.state()[2]).sum(0)
    hs = sc.sim.dt / sc.sim.n_substeps
    n_contacts = 0
    for _ in range(3):
        w.collide()
        ab, _ = w.pile_pairs(0)
        n_contacts += sum(len(w.pair_contacts(0, k)) for k in range(len(ab)))
        w.substep(hs, sc.sim.n_iters, detect=False)
    p1 = (m[:, None] * w.state()[2]).sum(0)
    assert n_contacts > 20
    v_change = np.abs(w.state()[2] - nb["linvel"]).max()
    assert v_change > 1e-3                                          # the contacts did act
    assert np.abs(p1 - p0).max() <= 1e-12 * m.sum() * max(1.0, np.abs(w.state()[2]).max()) * 100


def test_pile_of_resting_stacks_stays_at_rest():
    """Stacks apart from each other (no side contacts), each nut sunk 0.02 mm into its
    support: the pile env holds them as the listed-pair env does."""
    sc = S.nut_pile_env_scene(7, seed=1, mode="heap", n_samples=5000, sdf_res=128, plate_sdf_res=64,
                              overlap_mm=-3.0, n_substeps=8, n_iters=32, n_vel_iters=0)
    w = O.world_from_scene(sc, lazy_bake=True)
    p0 = w.state()[0].copy()
    for _ in range(10):
        w.step(sc.sim.n_substeps, sc.sim.n_iters)
    p, q, v, om = w.state()
    ab, col = w.pile_pairs(0)
    assert (col >= 0).sum() >= 7                                   # every nut rests on something
    assert np.abs(p[:-1] - p0[:-1]).max() <= 2e-4
    assert np.abs(v[:-1]).max() <= 2e-3 and np.abs(om[:-1]).max() <= 5e-2
    assert np.all(p[:-1, 2] > 0.0)
