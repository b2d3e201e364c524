"""FP16 SDF storage (phi / h in float16, interpolation and solve in float32) against the
float32 form and the FP64 oracle.

Bound used for the query: each stored corner is phi / h rounded to the nearest float16,
an error of at most 2^-11 |phi| (2^-25 h below the normal range); the trilinear value is
a convex combination of the corners, so it errs by at most 2^-11 max|corner phi| + 2^-25 h,
and each gradient component (a blend of corner differences over h) by twice that over h.
A small float32 term covers the interpolation's own rounding.

Pose accuracy: one frame of the 64 peg-in-hole envs around first contact, FP16 and FP32
worlds from the same inputs, each against the oracle; the test prints both errors.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


def _fw():
    from paper_2205_03532_b300 import fw
    return fw


def _corner_max(vals, lo, h, dims, pts):
    """max |phi| over the 8 corners of each point's cell (float64, numpy)"""
    u = (pts.astype(np.float64) - lo.astype(np.float64)) / np.float64(h)
    c = np.clip(np.floor(u).astype(np.int64), 0, dims.astype(np.int64) - 2)
    m = np.zeros(len(pts))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                m = np.maximum(m, np.abs(vals[c[:, 2] + dz, c[:, 1] + dy, c[:, 0] + dx].astype(np.float64)))
    return m


def test_fp16_query_within_rounding_bound_of_fp32():
    fw = _fw()
    sc = S.peg_in_hole_scene(n_envs=1, seed=0)
    hole = sc.assets[1]
    w32 = fw.World()
    a32 = w32.add_mesh_asset(hole.verts, hole.tris, None)
    w32.bake_sdf(a32, hole.sdf_res, hole.sdf_pad, True)
    lo, h, dims, vals = w32.get_sdf(a32)
    w16 = fw.World(sdf_fp16=1)
    a16 = w16.add_mesh_asset(hole.verts, hole.tris, None)
    w16.set_sdf(a16, lo, h, dims, vals)
    rng = np.random.default_rng(4)
    span = (dims - 1) * np.float64(h)
    pts = (lo + rng.uniform(0.0, 1.0, (100_000, 3)) * span).astype(np.float32)
    # half of them within two voxels of the surface, where contacts are decided
    near = np.argwhere(np.abs(vals) < 2 * h)
    pick = near[rng.integers(0, len(near), 50_000)]
    pts[:50_000] = (lo + (pick[:, ::-1] + rng.uniform(0, 1, (50_000, 3))) * np.float64(h)).astype(np.float32)
    p32, g32 = w32.query_sdf(a32, pts)
    p16, g16 = w16.query_sdf(a16, pts)
    ok = np.isfinite(p32)
    assert np.array_equal(ok, np.isfinite(p16)) and ok.mean() > 0.99
    cm = _corner_max(vals, lo, h, dims, pts[ok])
    bound = 2.0 ** -11 * cm + 2.0 ** -25 * h
    dphi = np.abs(p16[ok].astype(np.float64) - p32[ok])
    assert np.all(dphi <= bound + 1e-6 * h), float((dphi / (bound + 1e-6 * h)).max())
    dg = np.max(np.abs(g16[ok].astype(np.float64) - g32[ok]), axis=1)
    gbound = 2.0 * bound / h
    assert np.all(dg <= gbound + 1e-5), float((dg / (gbound + 1e-5)).max())
    # against the oracle's FP64 interpolation of the same float32 grid
    ophi, _, valid = O.query(vals.astype(np.float64), lo, h, dims, pts[ok])
    assert valid.all()
    d16 = np.abs(p16[ok] - ophi)
    assert np.all(d16 <= bound + 2e-5 * h)
    print(f"\nFP16 query: max |phi16 - phi32| = {dphi.max():.3e} m "
          f"({dphi.max() / h:.2e} h), near-surface max = {dphi[:50_000].max() / h:.2e} h; "
          f"max |phi16 - oracle| = {d16.max() / h:.2e} h; max |g16 - g32| = {dg.max():.2e}")


def _rot_angle(q1, q2):
    d = abs(float(np.dot(q1 / np.linalg.norm(q1), q2 / np.linalg.norm(q2))))
    return 2 * math.acos(min(1.0, d))


def _peg_scene():
    sc = S.peg_in_hole_scene(n_envs=64, seed=7)
    b = sc.groups[0].bodies
    rng = np.random.default_rng(7)
    b["pos"][:, 0, 2] = 12.5e-3 + rng.uniform(-4e-3, 0.3e-3, len(b))
    b["pos"][:, 0, :2] = rng.uniform(-0.09e-3, 0.09e-3, (len(b), 2))
    for e in range(len(b)):
        tilt = np.deg2rad(rng.uniform(-0.3, 0.3, 2))
        b["quat"][e, 0] = S.quat_mul(S.quat_axis_angle([1, 0, 0], tilt[0]), S.quat_axis_angle([0, 1, 0], tilt[1]))
    return sc


def test_fp16_frame_pose_accuracy_equals_fp32():
    fw = _fw()
    sc = _peg_scene()
    ow = O.world_from_scene(sc)
    errs = {}
    for fp16 in (False, True):
        gw = fw.world_from_scene(sc, fp16=fp16)
        p, q, v, w = gw.get_state()
        ow.set_state(p, q, v, w)
        gw.step(sc.sim.n_substeps, sc.sim.n_iters)
        ow.step(sc.sim.n_substeps, sc.sim.n_iters)
        gp, gq = gw.get_state()[:2]
        op, oq = ow.state()[:2]
        pegs = range(0, len(gp), 2)
        errs[fp16] = (max(float(np.linalg.norm(gp[i] - op[i])) for i in pegs),
                      max(_rot_angle(gq[i].astype(np.float64), oq[i]) for i in pegs))
        gw.close()
    print(f"\none frame, 64 peg envs vs the FP64 oracle: FP32 max pos {errs[False][0]:.2e} m, "
          f"rot {errs[False][1]:.2e} rad; FP16 max pos {errs[True][0]:.2e} m, rot {errs[True][1]:.2e} rad")
    # both forms within the frame tolerance used for envs with near-tie decisions
    for fp16 in (False, True):
        assert errs[fp16][0] <= 2e-4 and errs[fp16][1] <= 2e-3, (fp16, errs[fp16])
