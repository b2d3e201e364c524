"""The oracle's narrow-band bricked SDF storage (bricks of 8^3 cells kept when a node is
within the band or the nodes change sign; elsewhere a lookup answers +-band with no
gradient), pinned without its own classification code:

  * trilinear values are convex combinations of a cell's corners, so wherever the dense
    field has |phi| <= band the bricked lookup must return the dense value and gradient
    bit for bit; elsewhere it may only answer +band (outside) or -band (inside) with a
    zero gradient, never a value of the other sign;
  * on an analytic sphere field the number of stored bricks lies between two geometric
    counts: bricks whose node box the sphere crosses (each then has a node within
    sqrt(3)/2 h < band of the surface) and bricks whose node box comes within the band
    of the surface;
  * a world detects the same contacts with bricked and with dense storage while nothing
    penetrates deeper than the band (lazy bakes on both sides).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


def _sphere_grid(n=64, h=4e-4, r0=7e-3, c=(3e-4, -2e-4, 1e-4)):
    lo = np.full(3, -0.5 * (n - 1) * h, np.float32)
    i = lo[0] + np.arange(n) * np.float64(h)
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    vals = (np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) - r0).astype(np.float32)
    return lo, np.float32(h), np.array([n, n, n], np.int32), vals, np.array(c), r0


def _points(lo, h, n, c, r0, rng, k=40000):
    span = (n - 1) * float(h)
    a = lo + rng.uniform(0, span, (k, 3))                       # anywhere in the box
    d = rng.normal(size=(k, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    b = c + d * (r0 + rng.uniform(-4 * h, 4 * h, (k, 1)))      # near the surface
    return np.concatenate([a, b]).astype(np.float32)


@pytest.mark.parametrize("band", [2.0, 0.3])
def test_bricked_lookup_equals_dense_within_the_band(band):
    lo, h, dims, vals, c, r0 = _sphere_grid()
    pts = _points(lo, h, int(dims[0]), c, r0, np.random.default_rng(3))
    phi, grad, valid = O.query(vals.astype(np.float64), lo, h, dims, pts)
    bphi, bgrad, bvalid, ns, nb = O.query_band(vals.astype(np.float64), lo, h, dims, band, pts)
    assert np.array_equal(valid, bvalid)
    bw = np.float32(np.float32(band) * h)
    inb = valid & (np.abs(phi) <= bw)
    assert inb.sum() > 1000
    np.testing.assert_array_equal(bphi[inb], phi[inb])
    np.testing.assert_array_equal(bgrad[inb], grad[inb])
    diff = valid & ((bphi != phi) | np.any(bgrad != grad, axis=1))
    assert diff.sum() > 1000 and not np.any(diff & inb)
    assert np.all(np.abs(phi[diff]) > bw)
    np.testing.assert_array_equal(bphi[diff], np.where(phi[diff] > 0, float(bw), -float(bw)))
    np.testing.assert_array_equal(bgrad[diff], 0.0)
    assert 0 < ns < nb


def test_stored_brick_count_between_geometric_bounds():
    lo, h, dims, vals, c, r0 = _sphere_grid()
    band = 2.0
    _, _, _, ns, nb = O.query_band(vals.astype(np.float64), lo, h, dims, band, np.zeros((1, 3), np.float32))
    n = int(dims[0])
    nbx = (n - 1 + 7) // 8
    assert nb == nbx ** 3
    crossed = near = 0
    bw = band * float(h)
    for bk in range(nbx):
        for bj in range(nbx):
            for bi in range(nbx):
                b0 = np.array([bi, bj, bk]) * 8
                b1 = np.minimum(b0 + 8, n - 1)
                box_lo = lo.astype(np.float64) + b0 * float(h)
                box_hi = lo.astype(np.float64) + b1 * float(h)
                q = np.clip(c, box_lo, box_hi)                               # nearest box point to c
                dmin = np.linalg.norm(q - c)
                far = np.maximum(np.abs(box_lo - c), np.abs(box_hi - c))
                dmax = np.linalg.norm(far)
                crossed += int(dmin <= r0 <= dmax)
                near += int(dmin <= r0 + bw and dmax >= r0 - bw)
    assert crossed <= ns <= near, (crossed, ns, near)


def test_world_contacts_equal_with_bricked_storage():
    sc = S.peg_in_hole_scene(n_envs=6, seed=11)
    b = sc.groups[0].bodies
    b["pos"][:, 0, 2] = 12.5e-3 + np.linspace(-4e-3, 0.2e-3, 6)
    dense = O.world_from_scene(sc, lazy_bake=True)
    brick = O.world_from_scene(sc, lazy_bake=True, sdf_band=3.0)
    dense.collide()
    brick.collide()
    total = 0
    for env in range(sc.n_envs):
        a, _, _ = dense.contacts(env)
        c, _, _ = brick.contacts(env)
        assert list(a["sample"]) == list(c["sample"]) and list(a["patch"]) == list(c["patch"])
        np.testing.assert_array_equal(a["phi"], c["phi"])
        total += len(a)
    assert total > 50
    # the band is in force: samples far from the hole now have no gradient (no candidate)
    ns = len(sc.assets[0].samples)
    _, _, vd = dense.query_pair(0, 0, ns)
    _, _, vb = brick.query_pair(0, 0, ns)
    assert vb.sum() < vd.sum() and not np.any(vb & ~vd)
    dense.step(sc.sim.n_substeps, sc.sim.n_iters)
    brick.step(sc.sim.n_substeps, sc.sim.n_iters)
    for x, y in zip(dense.state(), brick.state()):
        np.testing.assert_array_equal(x, y)
