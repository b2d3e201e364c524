"""The bound the narrow phase's sample-group cull rests on (fw_set_query_cull; Sec. III-A
skips samples far from the other body): the SDF is a grid of signed distances (Sec. III-A),
so neighbouring nodes differ by at most one voxel h; the trilinear field between them then
changes by at most one per unit length along each axis, at most sqrt(3) in any direction,
and phi(x) >= phi(c) - sqrt(3) |x - c| for every x within reach of c inside the grid.  A
group of samples in a sphere (c, r) with phi(c) - 2.5 r > cutoff + h therefore holds no
sample below the cutoff.  Checked on the oracle's own bake and trilinear lookup of a torus
(curved everywhere) and a box with a hole (edges, a concave rim), at random centres and
radii of half a voxel to four voxels, points in each sphere and on its surface.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S

SQRT3 = np.sqrt(3.0)


def _grid(V, T, res):
    lo, h, dims = O.grid_params(V, res, 0.1)
    grid = O.bake_nodes(V, T, lo, h, dims)
    return grid, lo, float(h), dims


MESHES = {
    "torus": lambda: S.torus_mesh(0.02, 0.008, n_u=32, n_v=12),
    "box_with_hole": lambda: S.box_with_hole_mesh(0.04, 0.04, 0.02, 0.008, 0.015, 32),
}


@pytest.fixture(scope="module", params=sorted(MESHES))
def baked(request):
    V, T = MESHES[request.param]()
    return (request.param,) + _grid(np.asarray(V, np.float64), np.asarray(T), 24)


def test_neighbouring_nodes_differ_by_at_most_a_voxel(baked):
    """the premise: the baked nodes are distances, so one step along an axis changes phi by
    at most h (the exact distance is 1-Lipschitz; the bake is FP64)"""
    name, grid, lo, h, dims = baked
    g = grid  # (z, y, x)
    worst = max(np.abs(np.diff(g, axis=a)).max() for a in range(3))
    assert worst <= h * (1.0 + 1e-12), (name, worst / h)
    assert worst >= 0.5 * h, (name, worst / h)   # not a degenerate grid


def test_trilinear_field_falls_no_faster_than_sqrt3(baked):
    """phi(x) >= phi(c) - sqrt(3) |x - c| for points in and on random spheres"""
    name, grid, lo, h, dims = baked
    rng = np.random.default_rng(7)
    span = (dims.astype(np.float64) - 1.0) * h
    n_c, n_p = 400, 64
    r = rng.uniform(0.5, 4.0, n_c) * h
    c = lo + r[:, None] + rng.uniform(0.0, 1.0, (n_c, 3)) * (span - 2.0 * r[:, None])   # sphere inside the grid
    d = rng.normal(size=(n_c, n_p, 3))
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    rad = r[:, None] * np.concatenate([np.ones((n_c, n_p // 4)), rng.uniform(0.0, 1.0, (n_c, n_p - n_p // 4)) ** (1 / 3)],
                                      axis=1)
    x = (c[:, None, :] + d * rad[:, :, None]).astype(np.float32)
    cf = c.astype(np.float32)
    phi_c, _, ok_c = O.query(grid, lo, h, dims, cf)
    phi_x, _, ok_x = O.query(grid, lo, h, dims, x.reshape(-1, 3))
    assert ok_c.all() and ok_x.all()
    dist = np.linalg.norm(x.astype(np.float64) - cf.astype(np.float64)[:, None, :], axis=2).reshape(-1)
    drop = np.repeat(phi_c, n_p) - phi_x
    slack = SQRT3 * dist - drop
    assert slack.min() >= -1e-9 * h, (name, slack.min() / h)
    # the field does fall steeply somewhere: the bound is not vacuous here
    steep = (drop / np.maximum(dist, 1e-30))[dist > 0.25 * h]
    assert steep.max() > 0.9, (name, steep.max())


def test_a_culled_group_holds_no_candidate(baked):
    """the cull's rule: a sphere with phi(c) - 2.5 r > cutoff + h has every point above the
    cutoff (what the field can do over r, plus a voxel, with FP16 rounding room)"""
    name, grid, lo, h, dims = baked
    rng = np.random.default_rng(11)
    span = (dims.astype(np.float64) - 1.0) * h
    cutoff = 0.5 * h
    culled = 0
    for _ in range(300):
        r = rng.uniform(0.5, 4.0) * h
        c = lo + r + rng.uniform(0.0, 1.0, 3) * (span - 2.0 * r)
        phi_c = O.query(grid, lo, h, dims, c[None].astype(np.float32))[0][0]
        if not (phi_c - 2.5 * r > cutoff + h):
            continue
        culled += 1
        d = rng.normal(size=(128, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        x = (c + d * r * rng.uniform(0.0, 1.0, (128, 1)) ** (1 / 3)).astype(np.float32)
        phi_x, _, ok = O.query(grid, lo, h, dims, x)
        assert ok.all()
        assert phi_x.min() > cutoff, (name, phi_x.min() / h)
    assert culled >= 30, (name, culled)
