"""Narrow-band bricked SDF storage on the GPU (sdf_band > 0: bricks of 8^3 cells kept
within the band, lookups elsewhere answer +-band with no gradient) against the oracle's
reading of the same storage and against the GPU's own dense storage.

  * identical float32 grids: the bricked lookup against the oracle's bricked lookup with
    the dense tolerances (1e-5 h + 2^-21 |phi| in value, 1e-5 in gradient), and exactly
    +-band with a zero gradient where both leave the brick out (the decisions are taken
    on the same float32 node values, so they coincide); against the GPU's dense lookup
    bit for bit wherever |phi| <= band;
  * a whole frame of the nut-bolt and the peg scenes bit-identical to dense storage (no
    sample penetrates deeper than the band), in FP32 and in FP16, with the lookup copy
    far smaller than the dense one.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import oracle as O
from paper_2205_03532_b300 import scenes as S


def _fw():
    from paper_2205_03532_b300 import fw
    return fw


def _sphere(n=200, h=1.6e-4):
    lo = np.array([-0.016, -0.0155, -0.0162], np.float32)
    h = np.float32(h)
    i = np.arange(n, dtype=np.float64) * np.float64(h)
    Z, Y, X = np.meshgrid(i + lo[2], i + lo[1], i + lo[0], indexing="ij")
    vals = (np.sqrt(X * X + Y * Y + Z * Z) - 0.011 + 2e-4 * np.sin(900 * X) * np.cos(700 * Y)).astype(np.float32)
    return lo, h, np.array([n, n, n], np.int32), vals


@pytest.mark.parametrize("band", [3.0, 0.4])
def test_bricked_query_on_identical_grid(band):
    fw = _fw()
    lo, h, dims, vals = _sphere()
    V, T = S.box_mesh(0.01, 0.01, 0.01)
    wb, wd = fw.World(sdf_band=band), fw.World()
    ab, ad = wb.add_mesh_asset(V, T, None), wd.add_mesh_asset(V, T, None)
    wb.set_sdf(ab, lo, h, dims, vals)
    wd.set_sdf(ad, lo, h, dims, vals)
    rng = np.random.default_rng(5)
    span = (dims - 1) * np.float64(h)
    a = lo + rng.uniform(-0.02, 1.02, (150_000, 3)) * span
    d = rng.normal(size=(150_000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    b = d * (0.011 + rng.uniform(-6 * h, 6 * h, (150_000, 1)))
    pts = np.concatenate([a, b]).astype(np.float32)
    phi, grad = wb.query_sdf(ab, pts)
    dphi_, dgrad = wd.query_sdf(ad, pts)
    ophi, ograd, valid, ns, nb = O.query_band(vals.astype(np.float64), lo, h, dims, band, pts)
    assert np.array_equal(np.isfinite(phi), valid) and valid.sum() > 200_000
    bw = np.float32(np.float32(band) * h)
    out = valid & np.all(ograd == 0.0, axis=1) & (np.abs(ophi) == float(bw))
    inb = valid & ~out
    assert out.sum() > 10_000 and inb.sum() > 10_000
    # the oracle leaves these bricks out: so does the GPU, exactly
    np.testing.assert_array_equal(phi[out], ophi[out].astype(np.float32))
    np.testing.assert_array_equal(grad[out], 0.0)
    # stored bricks: the dense tolerances against the oracle
    dv = np.abs(phi[inb] - ophi[inb])
    assert np.all(dv <= 1e-5 * h + 2.0 ** -21 * np.abs(ophi[inb])), float(dv.max())
    dg = np.abs(grad[inb] - ograd[inb])
    assert np.all(dg <= 1e-5 * np.maximum(1.0, np.abs(ograd[inb]))), float(dg.max())
    # and bit for bit the GPU's dense lookup wherever |phi| <= band
    near = valid & (np.abs(dphi_) <= bw)
    np.testing.assert_array_equal(phi[near], dphi_[near])
    np.testing.assert_array_equal(grad[near], dgrad[near])
    nbytes, stored, total = wb.sdf_storage(ab)
    dbytes = wd.sdf_storage(ad)[0]
    assert (stored, total) == (ns, nb) and nbytes < dbytes
    wb.close()
    wd.close()


@pytest.mark.parametrize("scene,fp16", [("nut", False), ("nut", True), ("peg", False)])
def test_frame_bit_identical_to_dense(scene, fp16):
    fw = _fw()
    if scene == "nut":
        sc = S.nut_bolt_scene(n_envs=16, seed=4)
    else:
        sc = S.peg_in_hole_scene(n_envs=32, seed=8)
        b = sc.groups[0].bodies
        b["pos"][:, 0, 2] = 12.5e-3 + np.random.default_rng(8).uniform(-4e-3, 0.3e-3, len(b))
    wd = fw.world_from_scene(sc, fp16=fp16)
    wb = fw.world_from_scene(sc, fp16=fp16, sdf_band=4.0)
    for _ in range(2):
        wd.step(sc.sim.n_substeps, sc.sim.n_iters)
        wb.step(sc.sim.n_substeps, sc.sim.n_iters)
    for x, y in zip(wd.get_state(), wb.get_state()):
        np.testing.assert_array_equal(x, y)
    sdf_asset = 1
    dense, (brick, stored, total) = wd.sdf_storage(sdf_asset)[0], wb.sdf_storage(sdf_asset)
    assert 0 < stored < total
    print(f"{scene} fp16={fp16}: lookup copy {dense / 2**20:.1f} MiB dense, {brick / 2**20:.1f} MiB bricked "
          f"({stored} of {total} bricks)")
    # a 64^3 grid is only 8 bricks across, so the band keeps most of it; 256^3 keeps 1/7
    assert brick < (0.5 if scene == "nut" else 1.0) * dense
    wd.close()
    wb.close()
