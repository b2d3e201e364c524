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
