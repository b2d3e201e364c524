"""Seeded synthetic inputs: procedural meshes, surface sample points and initial poses.

This module builds the workloads only.  It holds none of the contact method's
arithmetic (no distance fields, no contact reduction, no solver, no mass
properties); both the CUDA path and the CPU oracle receive the arrays it makes.

Geometry follows the paper's scenes (Sec. IV-B, Table "geometric
representations"): a 4 mm-class peg and a box with a blind hole, ISO-metric
hex nuts and bolts with 60-degree threads and a small radial clearance, and
involute spur gears.  The paper's own CAD assets are not available, so these
procedural stand-ins take their shapes and sizes.

Conventions: metres, right-handed, z up, quaternions stored (x, y, z, w),
triangles wound counter-clockwise seen from outside (outward normal
(b - a) x (c - a)).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# body types (mirror of the C ABI's fw_body_type)
STATIC, KINEMATIC, DYNAMIC, FIXED_AXIS = 0, 1, 2, 3


# --------------------------------------------------------------------------------------
# mesh assembly helpers
# --------------------------------------------------------------------------------------
class _MeshBuilder:
    """Collects float64 vertices and triangles, then welds coincident vertices."""

    def __init__(self) -> None:
        self.pos: List[np.ndarray] = []
        self.tris: List[Tuple[int, int, int]] = []
        self.n = 0

    def add_vertices(self, p: np.ndarray) -> np.ndarray:
        p = np.asarray(p, dtype=np.float64).reshape(-1, 3)
        idx = np.arange(self.n, self.n + len(p))
        self.pos.append(p)
        self.n += len(p)
        return idx

    def add_tri(self, a: int, b: int, c: int) -> None:
        self.tris.append((int(a), int(b), int(c)))

    def add_tri_facing(self, a: int, b: int, c: int, outward: np.ndarray) -> None:
        """Adds (a, b, c) or (a, c, b), whichever has a normal along `outward`."""
        P = np.concatenate(self.pos) if len(self.pos) > 1 else self.pos[0]
        n = np.cross(P[b] - P[a], P[c] - P[a])
        if float(np.dot(n, outward)) < 0.0:
            b, c = c, b
        self.add_tri(a, b, c)

    def build(self, weld_tol: float = 1e-10) -> Tuple[np.ndarray, np.ndarray]:
        P = np.concatenate(self.pos)
        key = np.round(P / weld_tol).astype(np.int64)
        _, first, inverse = np.unique(key, axis=0, return_index=True, return_inverse=True)
        inverse = inverse.reshape(-1)
        T = inverse[np.asarray(self.tris, dtype=np.int64)]
        keep = (T[:, 0] != T[:, 1]) & (T[:, 1] != T[:, 2]) & (T[:, 0] != T[:, 2])
        T = T[keep]
        # renumber vertices in first-use order so that the layout is deterministic
        used, T_new = np.unique(T.reshape(-1), return_inverse=True)
        V = P[first[used]]
        T = T_new.reshape(-1, 3)
        V32 = V.astype(np.float32)
        T32 = T.astype(np.int32)
        area2 = np.linalg.norm(
            np.cross(V32[T32[:, 1]].astype(np.float64) - V32[T32[:, 0]],
                     V32[T32[:, 2]].astype(np.float64) - V32[T32[:, 0]]), axis=1)
        if np.any(area2 <= 0.0):
            raise ValueError("mesh has a zero-area triangle after welding")
        return V32, T32


def edge_manifold_check(T: np.ndarray) -> bool:
    """True iff every directed edge appears once and its reverse appears once
    (closed, consistently oriented 2-manifold edge structure)."""
    T = np.asarray(T, dtype=np.int64)
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    nv = int(T.max()) + 1
    fwd = e[:, 0] * nv + e[:, 1]
    rev = e[:, 1] * nv + e[:, 0]
    if len(np.unique(fwd)) != len(fwd):
        return False
    return bool(np.all(np.isin(rev, fwd)))


def signed_volume(V: np.ndarray, T: np.ndarray) -> float:
    """Enclosed volume (positive for outward winding); a mesh sanity check only."""
    V = np.asarray(V, dtype=np.float64)
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


# --------------------------------------------------------------------------------------
# simple closed meshes (used by pins and the peg scene)
# --------------------------------------------------------------------------------------
def box_mesh(hx: float, hy: float, hz: float) -> Tuple[np.ndarray, np.ndarray]:
    """Axis-aligned box [-hx,hx]x[-hy,hy]x[-hz,hz], 12 triangles."""
    mb = _MeshBuilder()
    c = np.array([[sx * hx, sy * hy, sz * hz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)])
    idx = mb.add_vertices(c)

    def vid(sx, sy, sz):
        return idx[((sx + 1) // 2) * 4 + ((sy + 1) // 2) * 2 + ((sz + 1) // 2)]

    for axis in range(3):
        for s in (-1, 1):
            quad = []
            for u, v in ((-1, -1), (1, -1), (1, 1), (-1, 1)):
                t = [0, 0, 0]
                t[axis] = s
                t[(axis + 1) % 3] = u
                t[(axis + 2) % 3] = v
                quad.append(vid(*t))
            out = np.zeros(3)
            out[axis] = s
            mb.add_tri_facing(quad[0], quad[1], quad[2], out)
            mb.add_tri_facing(quad[0], quad[2], quad[3], out)
    return mb.build()


def icosphere(r: float, level: int) -> Tuple[np.ndarray, np.ndarray]:
    """Subdivided icosahedron with all vertices on the sphere of radius r."""
    t = (1.0 + 5 ** 0.5) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
             (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    F = list(faces)
    for _ in range(level):
        cache = {}

        def mid(a, b):
            k = (min(a, b), max(a, b))
            if k not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[k] = len(V) - 1
            return cache[k]

        nf = []
        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = nf
    mb = _MeshBuilder()
    mb.add_vertices(np.array(V) * r)
    for a, b, c in F:
        mb.add_tri(a, b, c)
    return mb.build()


def cylinder_mesh(r: float, h: float, n_seg: int) -> Tuple[np.ndarray, np.ndarray]:
    """Closed n-gon prism of circumradius r along z, z in [-h/2, h/2], with
    centre vertices on both caps: 4*n_seg triangles (128 segments -> 512)."""
    mb = _MeshBuilder()
    th = 2.0 * np.pi * np.arange(n_seg) / n_seg
    ring = np.stack([r * np.cos(th), r * np.sin(th), np.zeros(n_seg)], 1)
    bot = mb.add_vertices(ring + [0, 0, -h / 2])
    top = mb.add_vertices(ring + [0, 0, h / 2])
    cb = mb.add_vertices([[0, 0, -h / 2]])[0]
    ct = mb.add_vertices([[0, 0, h / 2]])[0]
    for i in range(n_seg):
        j = (i + 1) % n_seg
        mb.add_tri(bot[i], bot[j], top[j])
        mb.add_tri(bot[i], top[j], top[i])
        mb.add_tri(ct, top[i], top[j])
        mb.add_tri(cb, bot[j], bot[i])
    return mb.build()


def torus_mesh(R: float, r: float, n_u: int = 64, n_v: int = 16) -> Tuple[np.ndarray, np.ndarray]:
    """Torus about the z axis: tube radius r around the circle of radius R in the xy plane;
    n_u segments around z, n_v around the tube (n_u n_v vertices, 2 n_u n_v triangles)."""
    mb = _MeshBuilder()
    th = 2.0 * np.pi * np.arange(n_u) / n_u
    ph = 2.0 * np.pi * np.arange(n_v) / n_v
    T, P = np.meshgrid(th, ph, indexing="ij")
    pts = np.stack([(R + r * np.cos(P)) * np.cos(T), (R + r * np.cos(P)) * np.sin(T), r * np.sin(P)], -1)
    idx = mb.add_vertices(pts.reshape(-1, 3)).reshape(n_u, n_v)
    for i in range(n_u):
        for j in range(n_v):
            a, b = idx[i, j], idx[(i + 1) % n_u, j]
            c, d = idx[(i + 1) % n_u, (j + 1) % n_v], idx[i, (j + 1) % n_v]
            tm, pm = 2.0 * np.pi * (i + 0.5) / n_u, 2.0 * np.pi * (j + 0.5) / n_v
            out = np.array([np.cos(pm) * np.cos(tm), np.cos(pm) * np.sin(tm), np.sin(pm)])   # tube normal
            mb.add_tri_facing(a, b, c, out)
            mb.add_tri_facing(a, c, d, out)
    return mb.build()


def bowl_mesh(rim: float, depth: float, wall: float, n_seg: int = 32, n_ring: int = 9) -> Tuple[np.ndarray, np.ndarray]:
    """A bowl: the shell between two concentric spherical caps (outer radius Ro, inner
    Ro - wall) cut by the rim plane, opening up: outer bottom at z = 0, rim at z = depth,
    outer rim radius `rim`.  Ro = (rim^2 + depth^2) / (2 depth).  Each cap is a pole vertex
    and n_ring rings of n_seg; the rim is the flat annulus between the caps' edges."""
    Ro = (rim * rim + depth * depth) / (2.0 * depth)
    Ri = Ro - wall
    c = np.array([0.0, 0.0, Ro])
    a_o = math.acos((Ro - depth) / Ro)
    a_i = math.acos((Ro - depth) / Ri)
    mb = _MeshBuilder()
    th = 2.0 * np.pi * np.arange(n_seg) / n_seg

    def cap(Rs, amax):
        pole = mb.add_vertices([c + [0.0, 0.0, -Rs]])[0]
        rings = []
        for k in range(1, n_ring + 1):
            a = amax * k / n_ring
            ring = np.stack([Rs * math.sin(a) * np.cos(th), Rs * math.sin(a) * np.sin(th),
                             np.full(n_seg, Ro - Rs * math.cos(a))], 1)
            rings.append(mb.add_vertices(ring))
        return pole, rings

    po, ro = cap(Ro, a_o)
    pi_, ri = cap(Ri, a_i)
    P = lambda i: np.concatenate(mb.pos)[i]
    for pole, rings, sign in ((po, ro, 1.0), (pi_, ri, -1.0)):   # outer faces away from c, inner towards it
        for i in range(n_seg):
            j = (i + 1) % n_seg
            q = rings[0]
            mb.add_tri_facing(pole, q[i], q[j], sign * ((P(q[i]) + P(q[j])) / 2 - c))
            for k in range(n_ring - 1):
                a, b = rings[k], rings[k + 1]
                mid = (P(a[i]) + P(a[j]) + P(b[i]) + P(b[j])) / 4 - c
                mb.add_tri_facing(a[i], a[j], b[j], sign * mid)
                mb.add_tri_facing(a[i], b[j], b[i], sign * mid)
    oe, ie = ro[-1], ri[-1]
    up = np.array([0.0, 0.0, 1.0])
    for i in range(n_seg):
        j = (i + 1) % n_seg
        mb.add_tri_facing(oe[i], oe[j], ie[j], up)
        mb.add_tri_facing(oe[i], ie[j], ie[i], up)
    return mb.build()


def _ray_square(th: np.ndarray, hx: float, hy: float) -> np.ndarray:
    c, s = np.cos(th), np.sin(th)
    t = np.minimum(np.where(np.abs(c) > 1e-15, hx / np.maximum(np.abs(c), 1e-300), np.inf),
                   np.where(np.abs(s) > 1e-15, hy / np.maximum(np.abs(s), 1e-300), np.inf))
    x, y = t * c, t * s
    # snap points that sit on a side exactly onto it (removes trig round-off at corners)
    x = np.where(np.isclose(np.abs(x), hx, rtol=0, atol=1e-12), np.sign(x) * hx, x)
    y = np.where(np.isclose(np.abs(y), hy, rtol=0, atol=1e-12), np.sign(y) * hy, y)
    return np.stack([x, y], 1)


def _ray_hexagon(th: np.ndarray, af: float) -> np.ndarray:
    """Ray/hexagon intersection; hexagon corners at angles 60k deg, across-flats af."""
    k = np.floor(th / (np.pi / 3) + 1e-9)
    mid = (k + 0.5) * (np.pi / 3)
    t = (af / 2) / np.cos(th - mid)
    return np.stack([t * np.cos(th), t * np.sin(th)], 1)


def _polygon_side_strips(mb: _MeshBuilder, top_ids, bot_ids, top_xy, z_top, z_bot):
    """Quad strip between two identical closed perimeters at z_top and z_bot; each
    triangle faces away from the axis (outward normal of a prism side)."""
    n = len(top_ids)
    for i in range(n):
        j = (i + 1) % n
        mid_xy = 0.5 * (top_xy[i] + top_xy[j])
        out = np.array([mid_xy[0], mid_xy[1], 0.0])
        mb.add_tri_facing(bot_ids[i], bot_ids[j], top_ids[j], out)
        mb.add_tri_facing(bot_ids[i], top_ids[j], top_ids[i], out)


def box_with_hole_mesh(sx: float, sy: float, sz: float, r: float, depth: float,
                       n_seg: int) -> Tuple[np.ndarray, np.ndarray]:
    """Box [-sx/2,sx/2]x[-sy/2,sy/2]x[-sz,0] with a blind cylindrical hole of radius r
    and the given depth opening on the top face (z = 0).  n_seg must be a multiple of 8
    so that rays through the square's corners are among the hole's rays."""
    assert n_seg % 8 == 0 and depth < sz
    mb = _MeshBuilder()
    th = 2.0 * np.pi * np.arange(n_seg) / n_seg
    circ = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    sq = _ray_square(th, sx / 2, sy / 2)
    c_top = mb.add_vertices(np.c_[circ, np.zeros(n_seg)])
    c_bot = mb.add_vertices(np.c_[circ, np.full(n_seg, -depth)])
    s_top = mb.add_vertices(np.c_[sq, np.zeros(n_seg)])
    hc = mb.add_vertices([[0, 0, -depth]])[0]
    up, down = np.array([0, 0, 1.0]), np.array([0, 0, -1.0])
    for i in range(n_seg):
        j = (i + 1) % n_seg
        # top annulus between hole rim and square outline
        mb.add_tri_facing(c_top[i], s_top[i], s_top[j], up)
        mb.add_tri_facing(c_top[i], s_top[j], c_top[j], up)
        # hole wall: the solid lies outside the hole, so faces point at the axis
        inward = -np.array([np.cos(th[i] + np.pi / n_seg), np.sin(th[i] + np.pi / n_seg), 0.0])
        mb.add_tri_facing(c_top[i], c_top[j], c_bot[j], inward)
        mb.add_tri_facing(c_top[i], c_bot[j], c_bot[i], inward)
        # hole bottom (solid below it, faces point up)
        mb.add_tri_facing(hc, c_bot[i], c_bot[j], up)
    # four side faces: fan from one bottom corner over the top-edge points
    hx, hy = sx / 2, sy / 2
    corners_b = {}
    for cx in (-1, 1):
        for cy in (-1, 1):
            corners_b[(cx, cy)] = mb.add_vertices([[cx * hx, cy * hy, -sz]])[0]
    for axis, sgn in ((0, 1), (1, 1), (0, -1), (1, -1)):
        coord = sq[:, axis]
        on = np.where(np.isclose(coord, sgn * (hx if axis == 0 else hy), atol=1e-12))[0]
        other = 1 - axis
        order = on[np.argsort(sq[on, other])]
        out = np.zeros(3)
        out[axis] = sgn
        if axis == 0:
            b0, b1 = corners_b[(sgn, -1)], corners_b[(sgn, 1)]
        else:
            b0, b1 = corners_b[(-1, sgn)], corners_b[(1, sgn)]
        pts = [s_top[k] for k in order]  # sorted along the other axis, from - to +
        mb.add_tri_facing(b0, b1, pts[-1], out)
        for k in range(len(pts) - 1, 0, -1):
            mb.add_tri_facing(b0, pts[k], pts[k - 1], out)
    # bottom face
    mb.add_tri_facing(corners_b[(-1, -1)], corners_b[(1, -1)], corners_b[(1, 1)], down)
    mb.add_tri_facing(corners_b[(-1, -1)], corners_b[(1, 1)], corners_b[(-1, 1)], down)
    return mb.build()


# --------------------------------------------------------------------------------------
# ISO-metric threads
# --------------------------------------------------------------------------------------
ISO_COARSE = {  # nominal d: (pitch, nut across-flats, nut thickness) in mm
    8: (1.25, 13.0, 6.8),
    12: (1.75, 18.0, 10.8),
    16: (2.0, 24.0, 13.0),
    20: (2.5, 30.0, 18.0),
}


def iso_basic_profile(d: float, P: float) -> np.ndarray:
    """Radii of the ISO 68-1 basic external-thread profile at the 16 phases s = j/16
    of one pitch: crest flat P/8 (2 steps), falling flank 5P/16 (5 steps), root flat
    P/4 (4 steps), rising flank 5P/16 (5 steps).  Depth 5H/8, H = sqrt(3)/2 P."""
    R = d / 2
    depth = 5.0 / 8.0 * (np.sqrt(3) / 2) * P
    r = np.empty(16)
    for j in range(16):
        if j <= 2:
            r[j] = R
        elif j <= 7:
            r[j] = R - depth * (j - 2) / 5.0
        elif j <= 11:
            r[j] = R - depth
        else:
            r[j] = R - depth * (16 - j) / 5.0
    return r


def _thread_surface(mb: _MeshBuilder, prof: np.ndarray, P: float, n_ang: int,
                    z_lo: float, z_hi: float, r_end: float, ramp: float,
                    inward: bool):
    """Helical surface r = prof(frac(z/P - theta/2pi)) between the planes z_lo and z_hi.

    Vertices sit on a sheared grid: angle index i (n_ang per turn) and profile row j
    (16 per pitch) at z = P (j + 16 i / n_ang) / 16, so profile kinks lie exactly on
    grid lines.  The thread depth fades to r_end over `ramp` at both ends, and vertices
    beyond an end plane are clamped onto it; since they all have radius r_end they weld
    into the rim circle, leaving only degenerate triangles (dropped by the builder).
    Returns the vertex ids of the rim circles at z_lo and z_hi (index = angle index)."""
    j_min = int(math.floor(z_lo * 16 / P)) - 17
    j_max = int(math.ceil(z_hi * 16 / P)) + 2
    rows = j_max - j_min + 1
    ids = np.empty((n_ang + 1, rows), dtype=np.int64)
    th = 2.0 * np.pi * (np.arange(n_ang + 1) % n_ang) / n_ang
    for i in range(n_ang + 1):
        j = np.arange(j_min, j_max + 1)
        z = P * (j * n_ang + 16 * i) / (16.0 * n_ang)
        w = np.clip((z - z_lo) / ramp, 0, 1) * np.clip((z_hi - z) / ramp, 0, 1)
        r = r_end + (prof[np.mod(j, 16)] - r_end) * w
        zc = np.clip(z, z_lo, z_hi)
        pts = np.stack([r * np.cos(th[i]), r * np.sin(th[i]), zc], 1)
        ids[i] = mb.add_vertices(pts)
    for i in range(n_ang):
        for jj in range(rows - 1):
            a, b, c, d = ids[i, jj], ids[i + 1, jj], ids[i + 1, jj + 1], ids[i, jj + 1]
            if inward:
                mb.add_tri(a, c, b)
                mb.add_tri(a, d, c)
            else:
                mb.add_tri(a, b, c)
                mb.add_tri(a, c, d)
    rim = np.stack([r_end * np.cos(th[:n_ang]), r_end * np.sin(th[:n_ang])], 1)
    lo_ids = mb.add_vertices(np.c_[rim, np.full(n_ang, z_lo)])
    hi_ids = mb.add_vertices(np.c_[rim, np.full(n_ang, z_hi)])
    return lo_ids, hi_ids, rim


def bolt_mesh(d_mm: float = 16.0, P_mm: float = 2.0, thread_len_mm: float = 30.0,
              head_af_mm: float = 24.0, head_h_mm: float = 10.0, n_ang: int = 42):
    """ISO hex bolt: hex head z in [-head_h, 0], threaded shank z in [0, thread_len].
    The thread fades to the root radius over half a pitch at both ends."""
    assert n_ang % 6 == 0
    s = 1e-3
    P, d = P_mm * s, d_mm * s
    prof = iso_basic_profile(d, P)
    r_root = float(prof.min())
    mb = _MeshBuilder()
    L = thread_len_mm * s
    lo_ids, hi_ids, rim = _thread_surface(mb, prof, P, n_ang, 0.0, L, r_root, P / 2, False)
    up, down = np.array([0, 0, 1.0]), np.array([0, 0, -1.0])
    ct = mb.add_vertices([[0, 0, L]])[0]
    for i in range(n_ang):
        j = (i + 1) % n_ang
        mb.add_tri_facing(ct, hi_ids[i], hi_ids[j], up)
    th = 2.0 * np.pi * np.arange(n_ang) / n_ang
    hexp = _ray_hexagon(th, head_af_mm * s)
    H = head_h_mm * s
    h_top = mb.add_vertices(np.c_[hexp, np.zeros(n_ang)])
    h_bot = mb.add_vertices(np.c_[hexp, np.full(n_ang, -H)])
    cb = mb.add_vertices([[0, 0, -H]])[0]
    for i in range(n_ang):
        j = (i + 1) % n_ang
        mb.add_tri_facing(lo_ids[i], h_top[i], h_top[j], up)
        mb.add_tri_facing(lo_ids[i], h_top[j], lo_ids[j], up)
        mb.add_tri_facing(cb, h_bot[j], h_bot[i], down)
    _polygon_side_strips(mb, h_top, h_bot, hexp, 0.0, -H)
    return mb.build()


def nut_mesh(d_mm: float = 16.0, P_mm: float = 2.0, thick_mm: float = 13.0,
             af_mm: float = 24.0, clearance_mm: float = 0.05, n_ang: int = 84):
    """ISO hex nut centred at the origin, z in [-thick/2, thick/2].  Its internal thread
    is the basic profile offset radially by +clearance; the thread depth fades to the
    root radius over half a pitch at both faces (a countersink stand-in).  The helix
    phase matches bolt_mesh: a nut at yaw psi meshes with the bolt at z = kP + P psi/2pi."""
    assert n_ang % 6 == 0
    s = 1e-3
    P, d = P_mm * s, d_mm * s
    prof = iso_basic_profile(d, P) + clearance_mm * s
    r_end = float(prof.max())
    T = thick_mm * s
    mb = _MeshBuilder()
    lo_ids, hi_ids, rim = _thread_surface(mb, prof, P, n_ang, -T / 2, T / 2, r_end, P / 2, True)
    th = 2.0 * np.pi * np.arange(n_ang) / n_ang
    hexp = _ray_hexagon(th, af_mm * s)
    up, down = np.array([0, 0, 1.0]), np.array([0, 0, -1.0])
    h_top = mb.add_vertices(np.c_[hexp, np.full(n_ang, T / 2)])
    h_bot = mb.add_vertices(np.c_[hexp, np.full(n_ang, -T / 2)])
    for i in range(n_ang):
        j = (i + 1) % n_ang
        mb.add_tri_facing(hi_ids[i], h_top[i], h_top[j], up)
        mb.add_tri_facing(hi_ids[i], h_top[j], hi_ids[j], up)
        mb.add_tri_facing(lo_ids[i], h_bot[j], h_bot[i], down)
        mb.add_tri_facing(lo_ids[i], lo_ids[j], h_bot[j], down)
    _polygon_side_strips(mb, h_top, h_bot, hexp, T / 2, -T / 2)
    return mb.build()


# --------------------------------------------------------------------------------------
# involute spur gears
# --------------------------------------------------------------------------------------
def gear_outline(module_mm: float, teeth: int, backlash_mm: float, n_flank: int = 24,
                 n_tip: int = 6, n_root: int = 8) -> np.ndarray:
    """Closed CCW outline (metres) of a 20-degree involute spur gear: per tooth the
    root arc, rising involute flank, tip arc and falling flank.  The tooth is thinned
    by backlash/2 of arc length on the pitch circle (half the pair's backlash each)."""
    s = 1e-3
    m = module_mm * s
    alpha = np.deg2rad(20.0)
    rp = m * teeth / 2
    rb = rp * np.cos(alpha)
    ra = rp + m
    rf = max(rp - 1.25 * m, 0.5 * rb)
    inv = lambda a: np.tan(a) - a
    half_tooth = (np.pi * m / 2 - backlash_mm * s / 2) / (2 * rp)  # half-angle at pitch
    phi_p = inv(alpha)
    pts = []
    pitch_ang = 2 * np.pi / teeth
    r_start = max(rb, rf)
    for k in range(teeth):
        c = k * pitch_ang
        # flank radii from the base (or root) circle to the tip circle
        rr = np.linspace(r_start, ra, n_flank)
        a_r = np.arccos(np.clip(rb / rr, -1, 1))
        off = half_tooth + phi_p - inv(a_r)  # angle of the flank point from the tooth axis
        left = np.stack([rr, c - off], 1)  # rising flank (angle increasing toward axis)
        right = np.stack([rr[::-1], c + off[::-1]], 1)
        tip_a = np.linspace(c - off[-1], c + off[-1], n_tip + 2)[1:-1]
        tip = np.stack([np.full_like(tip_a, ra), tip_a], 1)
        nxt = c + pitch_ang
        root_a = np.linspace(c + off[0], nxt - off[0], n_root + 2)
        root_a = root_a[1:-1]
        root = np.stack([np.full_like(root_a, rf), root_a], 1)
        seg = [left, tip, right]
        # below the base circle the flank drops to the root circle along a line turned a
        # quarter of a root step off the radius (a radial drop would put two outline
        # points on one ray, and the caps are triangulated along rays)
        dr = 0.25 * (nxt - c - 2 * off[0]) / (n_root + 1)
        if rf < r_start - 1e-12:
            seg.append(np.array([[rf, c + off[0] + dr]]))
        seg.append(root)
        if rf < r_start - 1e-12:
            seg.append(np.array([[rf, nxt - off[0] - dr]]))
        pts.append(np.concatenate(seg))
    polar = np.concatenate(pts)
    return np.stack([polar[:, 0] * np.cos(polar[:, 1]), polar[:, 0] * np.sin(polar[:, 1])], 1)


def gear_mesh(module_mm: float = 1.0, teeth: int = 20, thick_mm: float = 10.0,
              backlash_mm: float = 0.1, bore_mm: Optional[float] = None,
              n_flank: int = 24, n_tip: int = 6, n_root: int = 8, n_layers: int = 1):
    """Extruded involute spur gear, z in [-thick/2, thick/2], with a central bore.
    Faces: tooth outline strip(s), bore strip, and annular caps triangulated by
    matching every outline point with the bore point on the same ray."""
    s = 1e-3
    out = gear_outline(module_mm, teeth, backlash_mm, n_flank, n_tip, n_root)
    n = len(out)
    rf = float(np.min(np.linalg.norm(out, axis=1)))
    rb = (bore_mm * s / 2) if bore_mm else 0.35 * rf
    ang = np.arctan2(out[:, 1], out[:, 0])
    bore = np.stack([rb * np.cos(ang), rb * np.sin(ang)], 1)
    T = thick_mm * s
    mb = _MeshBuilder()
    zs = np.linspace(-T / 2, T / 2, n_layers + 1)
    o_ids = [mb.add_vertices(np.c_[out, np.full(n, z)]) for z in zs]
    b_ids = [mb.add_vertices(np.c_[bore, np.full(n, z)]) for z in zs]
    up, down = np.array([0, 0, 1.0]), np.array([0, 0, -1.0])
    for L in range(n_layers):
        for i in range(n):
            j = (i + 1) % n
            e = out[j] - out[i]
            nrm = np.array([e[1], -e[0], 0.0])  # CCW outline: right-hand normal is outward
            mb.add_tri_facing(o_ids[L][i], o_ids[L][j], o_ids[L + 1][j], nrm)
            mb.add_tri_facing(o_ids[L][i], o_ids[L + 1][j], o_ids[L + 1][i], nrm)
            cin = -np.array([bore[i][0] + bore[j][0], bore[i][1] + bore[j][1], 0.0])
            mb.add_tri_facing(b_ids[L][i], b_ids[L][j], b_ids[L + 1][j], cin)
            mb.add_tri_facing(b_ids[L][i], b_ids[L + 1][j], b_ids[L + 1][i], cin)
    for i in range(n):
        j = (i + 1) % n
        mb.add_tri_facing(b_ids[-1][i], o_ids[-1][i], o_ids[-1][j], up)
        mb.add_tri_facing(b_ids[-1][i], o_ids[-1][j], b_ids[-1][j], up)
        mb.add_tri_facing(b_ids[0][i], o_ids[0][j], o_ids[0][i], down)
        mb.add_tri_facing(b_ids[0][i], b_ids[0][j], o_ids[0][j], down)
    return mb.build()


# --------------------------------------------------------------------------------------
# surface samples, poses
# --------------------------------------------------------------------------------------
def _morton_key(q: np.ndarray) -> np.ndarray:
    """Interleaves three 10-bit integer coordinates into a 30-bit Morton code."""
    def spread(v):
        v = v.astype(np.uint64) & np.uint64(0x3FF)
        v = (v | (v << np.uint64(16))) & np.uint64(0x030000FF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x0300F00F)
        v = (v | (v << np.uint64(4))) & np.uint64(0x030C30C3)
        v = (v | (v << np.uint64(2))) & np.uint64(0x09249249)
        return v
    return spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1)) | (spread(q[:, 2]) << np.uint64(2))


def sample_surface(V: np.ndarray, T: np.ndarray, n: int, rng: np.random.Generator,
                   morton: bool = True) -> np.ndarray:
    """n points uniform by area on the mesh (triangle by area CDF, then the
    square-root barycentric map of Osada et al. 2002), sorted along a Morton curve of
    the mesh bounding box so that neighbouring indices are neighbouring in space."""
    V = np.asarray(V, dtype=np.float64)
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    cdf = np.cumsum(area)
    cdf /= cdf[-1]
    t = np.searchsorted(cdf, rng.random(n), side="right")
    t = np.minimum(t, len(T) - 1)
    r1 = np.sqrt(rng.random(n))[:, None]
    r2 = rng.random(n)[:, None]
    p = (1 - r1) * a[t] + r1 * (1 - r2) * b[t] + r1 * r2 * c[t]
    if morton:
        lo, hi = V.min(0), V.max(0)
        q = np.floor((p - lo) / np.maximum(hi - lo, 1e-30) * 1023.999).astype(np.int64)
        order = np.argsort(_morton_key(np.clip(q, 0, 1023)), kind="stable")
        p = p[order]
    return p.astype(np.float32)


def quat_axis_angle(axis, angle) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    s = math.sin(angle / 2)
    return np.array([axis[0] * s, axis[1] * s, axis[2] * s, math.cos(angle / 2)])


def quat_mul(a, b) -> np.ndarray:
    ax, ay, az, aw = a
    bx, by, bz, bw = b
    return np.array([aw * bx + bw * ax + ay * bz - az * by,
                     aw * by + bw * ay + az * bx - ax * bz,
                     aw * bz + bw * az + ax * by - ay * bx,
                     aw * bw - ax * bx - ay * by - az * bz])


# --------------------------------------------------------------------------------------
# scene containers
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class Asset:
    name: str
    verts: np.ndarray                 # float32 (nv, 3)
    tris: np.ndarray                  # int32 (nt, 3)
    samples: Optional[np.ndarray]     # float32 (ns, 3) or None
    density: float
    sdf_res: Optional[int] = None     # voxels on the longest axis (None: no SDF)
    sdf_pad: float = 1e-3


BODY_DTYPE = np.dtype([
    ("asset", np.int32), ("type", np.int32), ("mass", np.float32), ("mu", np.float32),
    ("pos", np.float32, 3), ("quat", np.float32, 4), ("linvel", np.float32, 3),
    ("angvel", np.float32, 3), ("axis", np.float32, 3), ("force", np.float32, 3),
    ("torque", np.float32, 3)])


@dataclasses.dataclass
class EnvGroup:
    """n_envs environments sharing one body/pair structure."""
    bodies: np.ndarray                # BODY_DTYPE (n_envs, n_per_env)
    pairs: np.ndarray                 # int32 (n_pairs, 2): (point body a, SDF body b), local ids


@dataclasses.dataclass
class SimParams:
    dt: float = 1.0 / 60.0
    n_substeps: int = 4
    n_iters: int = 16
    frames: int = 120
    gravity: Tuple[float, float, float] = (0.0, 0.0, -9.81)
    contact_offset: float = 1e-4
    cos_patch: float = 0.94
    max_patches: int = 128
    batch_size: int = 1024
    baumgarte: float = 0.2
    n_vel_iters: int = 0
    max_angvel: float = 0.0


@dataclasses.dataclass
class Scene:
    name: str
    assets: List[Asset]
    groups: List[EnvGroup]
    sim: SimParams
    # pile envs: BODY_DTYPE (n_bodies,) each; their pairs are found at every detection.
    # They follow the groups' envs in env order.
    piles: List[np.ndarray] = dataclasses.field(default_factory=list)

    @property
    def n_envs(self) -> int:
        return sum(g.bodies.shape[0] for g in self.groups) + len(self.piles)


def _body(asset, btype, pos, quat, mu, mass=0.0, linvel=(0, 0, 0), angvel=(0, 0, 0),
          axis=(0, 0, 1), force=(0, 0, 0), torque=(0, 0, 0)):
    b = np.zeros((), dtype=BODY_DTYPE)
    b["asset"], b["type"], b["mass"], b["mu"] = asset, btype, mass, mu
    b["pos"], b["quat"] = pos, quat
    b["linvel"], b["angvel"], b["axis"] = linvel, angvel, axis
    b["force"], b["torque"] = force, torque
    return b


def peg_in_hole_scene(n_envs: int = 1, seed: int = 0, clearance_mm: float = 0.1,
                      n_samples: int = 2000, sdf_res: int = 64,
                      n_substeps: int = 4, n_iters: int = 16, frames: int = 120,
                      mu: float = 0.5, mass_range_g: Optional[Tuple[float, float]] = None,
                      mu_range: Optional[Tuple[float, float]] = None) -> Scene:
    """Cylinder peg (r 4 mm, 25 mm, 512 triangles, 2,000 samples) dropped from 2 mm
    above a 24x24x16 mm box with a blind hole (r = 4 mm + clearance, depth 12 mm,
    168 segments -> 1,014 triangles) whose SDF is baked on a 64^3 grid with 1 mm
    padding.  Per env: lateral offset ~U(-0.3, 0.3) mm, tilts about x and y
    ~U(-2, 2) deg.  The box is static; the peg is dynamic."""
    rng = np.random.default_rng(seed)
    peg_V, peg_T = cylinder_mesh(4e-3, 25e-3, 128)
    hole_V, hole_T = box_with_hole_mesh(24e-3, 24e-3, 16e-3, 4e-3 + clearance_mm * 1e-3, 12e-3, 168)
    peg = Asset("peg", peg_V, peg_T, sample_surface(peg_V, peg_T, n_samples, rng), 7800.0)
    hole = Asset("hole", hole_V, hole_T, None, 7800.0, sdf_res=sdf_res, sdf_pad=1e-3)
    bodies = np.zeros((n_envs, 2), dtype=BODY_DTYPE)
    for e in range(n_envs):
        off = rng.uniform(-0.3e-3, 0.3e-3, 2)
        tx, ty = np.deg2rad(rng.uniform(-2, 2, 2))
        q = quat_mul(quat_axis_angle([1, 0, 0], tx), quat_axis_angle([0, 1, 0], ty))
        m = 0.0 if mass_range_g is None else rng.uniform(*mass_range_g) * 1e-3
        mu_e = mu if mu_range is None else rng.uniform(*mu_range)
        bodies[e, 0] = _body(0, DYNAMIC, (off[0], off[1], 2e-3 + 12.5e-3), q, mu_e, mass=m)
        bodies[e, 1] = _body(1, STATIC, (0, 0, 0), (0, 0, 0, 1), mu_e)
    pairs = np.array([[0, 1]], dtype=np.int32)
    sim = SimParams(n_substeps=n_substeps, n_iters=n_iters, frames=frames)
    return Scene("peg_in_hole", [peg, hole], [EnvGroup(bodies, pairs)], sim)


def diff_peg_scene(n_envs: int = 256, seed: int = 0, n_substeps: int = 32, n_iters: int = 8,
                   mass_range_g: Tuple[float, float] = (5.0, 50.0),
                   mu_range: Tuple[float, float] = (0.2, 0.8)) -> Tuple[Scene, np.ndarray, np.ndarray]:
    """Differentiable peg-in-hole: the peg-in-hole geometry with 0.1 mm clearance, one
    frame of 32 substeps x 8 sweeps, peg mass ~U(5, 50) g and friction ~U(0.2, 0.8) per
    env.  Each peg starts 1-3 mm into the hole (the rollout is in contact throughout),
    offset up to 0.08 mm sideways, tilted up to 0.3 deg, moving down at 2 cm/s with a
    small sideways velocity and spin, pressed down by a constant 0.5 N (a gripper pushing
    it in: without an applied force the motion under gravity and rigid contacts does not
    depend on the mass, whose gradient would then be zero).  Returns the scene and
    per-env target poses (peg bottom 6 mm into the hole, upright, centred) for a
    squared-distance loss.""" 
    sc = peg_in_hole_scene(n_envs=n_envs, seed=seed, clearance_mm=0.1, n_substeps=n_substeps,
                           n_iters=n_iters, frames=1, mass_range_g=mass_range_g, mu_range=mu_range)
    b = sc.groups[0].bodies
    rng = np.random.default_rng(seed + 1)
    b["pos"][:, 0, 2] = 12.5e-3 - rng.uniform(1e-3, 3e-3, n_envs)
    b["pos"][:, 0, :2] = rng.uniform(-0.08e-3, 0.08e-3, (n_envs, 2))
    b["linvel"][:, 0] = np.stack([rng.uniform(-5e-3, 5e-3, n_envs), rng.uniform(-5e-3, 5e-3, n_envs),
                                  np.full(n_envs, -0.02)], axis=1)
    b["angvel"][:, 0] = rng.uniform(-0.5, 0.5, (n_envs, 3))
    b["force"][:, 0] = [0.0, 0.0, -0.5]
    for e in range(n_envs):
        t = np.deg2rad(rng.uniform(-0.3, 0.3, 2))
        b["quat"][e, 0] = quat_mul(quat_axis_angle([1, 0, 0], t[0]), quat_axis_angle([0, 1, 0], t[1]))
    target_pos = np.zeros((n_envs, 3))
    target_pos[:, 2] = 12.5e-3 - 6e-3
    target_quat = np.tile([0.0, 0.0, 0.0, 1.0], (n_envs, 1))
    return sc, target_pos, target_quat


def nut_bolt_assets(d: int = 16, n_samples: int = 10000, sdf_res: int = 256,
                    rng: Optional[np.random.Generator] = None, clearance_mm: float = 0.05,
                    bolt_n_ang: int = 42, nut_n_ang: int = 84):
    P, af, thick = ISO_COARSE[d]
    if d == 16:
        thick = 13.0
    rng = rng or np.random.default_rng(0)
    bV, bT = bolt_mesh(d, P, thread_len_mm=15 * P, head_af_mm=af, head_h_mm=10.0 * d / 16,
                       n_ang=bolt_n_ang)
    nV, nT = nut_mesh(d, P, thick, af, clearance_mm, n_ang=nut_n_ang)
    nut = Asset(f"nut_m{d}", nV, nT, sample_surface(nV, nT, n_samples, rng), 7800.0)
    bolt = Asset(f"bolt_m{d}", bV, bT, None, 7800.0, sdf_res=sdf_res, sdf_pad=1e-3)
    return nut, bolt, P * 1e-3, thick * 1e-3, 15 * P * 1e-3


def nut_bolt_scene(n_envs: int = 1000, seed: int = 0, d: int = 16, n_samples: int = 10000,
                   sdf_res: int = 256, n_substeps: int = 8, n_iters: int = 32,
                   frames: int = 600, torque: float = 0.1, mu: float = 0.05,
                   bolt_n_ang: int = 42, nut_n_ang: int = 84) -> Scene:
    """Procedural ISO M16 nut on bolt (pitch 2 mm, 60-degree thread, 0.05 mm radial
    clearance); one SDF per bolt shared by all envs; 10k samples on the nut.  The nut
    starts engaged (its lower face about two pitches below the bolt tip, about one
    full turn of thread in mesh once the end fades are discounted) with yaw
    psi ~U(0, 60) deg and z = kP + P psi / 2pi so that the threads mesh without
    overlap; a tightening torque (-torque about +z, right-hand thread) is applied."""
    rng = np.random.default_rng(seed)
    nut, bolt, P, thick, L = nut_bolt_assets(d, n_samples, sdf_res, rng, bolt_n_ang=bolt_n_ang, nut_n_ang=nut_n_ang)
    bodies = np.zeros((n_envs, 2), dtype=BODY_DTYPE)
    k = int(math.floor((L - 2 * P + thick / 2) / P))
    for e in range(n_envs):
        psi = np.deg2rad(rng.uniform(0.0, 60.0))
        z = k * P + P * psi / (2 * np.pi)
        bodies[e, 0] = _body(0, DYNAMIC, (0, 0, z), quat_axis_angle([0, 0, 1], psi), mu,
                             torque=(0, 0, -torque))
        bodies[e, 1] = _body(1, STATIC, (0, 0, 0), (0, 0, 0, 1), mu)
    sim = SimParams(n_substeps=n_substeps, n_iters=n_iters, frames=frames, max_angvel=100.0)
    return Scene("nut_bolt", [nut, bolt], [EnvGroup(bodies, np.array([[0, 1]], np.int32))], sim)


# per size: SDF resolution (voxels on the longest axis) and samples on the nut
MIXED_NUT_BOLT = {8: (128, 5000), 12: (176, 10000), 16: (224, 20000), 20: (256, 40000)}


def mixed_nut_bolt_scene(n_envs: int = 4096, seed: int = 0, n_substeps: int = 8, n_iters: int = 32,
                         frames: int = 1) -> Scene:
    """Batched uneven environments: M8 / M12 / M16 / M20 nut-on-bolt pairs drawn uniformly
    by seed, SDF resolutions 128^3 - 256^3 and 5k - 40k samples per nut
    (MIXED_NUT_BOLT); angular segments of the threads scale with the diameter (multiples
    of 6 for the hex: 24/48 for M8 ... 54/108 for M20) so the chord error stays near half
    the clearance.  The drive torque scales with the nut's size, 0.1 N m (d/16)^3, so that
    every size turns at a comparable rate.  Envs of one size are contiguous (one group per
    size)."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(sorted(MIXED_NUT_BOLT), n_envs)
    assets: List[Asset] = []
    groups: List[EnvGroup] = []
    sim = None
    for d in sorted(MIXED_NUT_BOLT):
        n_d = int((sizes == d).sum())
        if n_d == 0:
            continue
        res, ns = MIXED_NUT_BOLT[d]
        sub = nut_bolt_scene(n_envs=n_d, seed=seed + d, d=d, n_samples=ns, sdf_res=res, n_substeps=n_substeps,
                             n_iters=n_iters, frames=frames, torque=0.1 * (d / 16.0) ** 3,
                             bolt_n_ang=6 * max(4, round(7 * d / 16)),
                             nut_n_ang=6 * max(7, round(14 * d / 16)))
        b = sub.groups[0].bodies.copy()
        b["asset"] += len(assets)
        assets += sub.assets
        groups.append(EnvGroup(b, sub.groups[0].pairs))
        sim = sub.sim
    return Scene("mixed_nut_bolt", assets, groups, sim)



GEAR_TEETH = (20, 30, 40)


def gear_assets(module_mm: float = 1.0, teeth: Sequence[int] = GEAR_TEETH, thick_mm: float = 10.0,
                backlash_mm: float = 0.1, tri_target: int = 30000, n_samples: int = 15000,
                sdf_res: int = 256, rng: Optional[np.random.Generator] = None) -> List[Asset]:
    """One asset per gear of the train: extruded in as many layers as bring it near
    tri_target triangles, n_samples surface samples on every gear that is a pair's point
    body (all but the last) and an SDF on every gear that is a pair's SDF body (all but
    the first)."""
    rng = rng or np.random.default_rng(0)
    assets = []
    for i, z in enumerate(teeth):
        n_out = len(gear_outline(module_mm, z, backlash_mm))
        layers = max(1, int(round(tri_target / (4.0 * n_out))) - 1)
        V, T = gear_mesh(module_mm, z, thick_mm, backlash_mm, n_layers=layers)
        samples = sample_surface(V, T, n_samples, rng) if i < len(teeth) - 1 else None
        assets.append(Asset(f"gear_z{z}", V, T, samples, 7800.0,
                            sdf_res=sdf_res if i > 0 else None, sdf_pad=1e-3))
    return assets


def gear_scene(n_envs: int = 2048, seed: int = 0, module_mm: float = 1.0, backlash_mm: float = 0.1,
               tri_target: int = 30000, n_samples: int = 15000, sdf_res: int = 256,
               drive_rate: float = 2.0, load_torque: float = 0.02, mu: float = 0.1,
               n_substeps: int = 8, n_iters: int = 32, frames: int = 300) -> Scene:
    """Gear train: involute spur gears of 20, 30 and 40 teeth (module 1 mm, 10 mm thick,
    0.1 mm backlash per mesh) on fixed parallel shafts along +z, in a row along +x at the
    standard centre distances m (z1 + z2) / 2.  The 20-tooth gear is kinematic, driven at
    drive_rate rad/s about +z; the 30- and 40-tooth gears are fixed-axis bodies free to
    spin about their shafts, the last one loaded by a constant torque against its turning
    direction (so that the flanks stay in contact).  Pairs: the samples of the smaller
    gear against the SDF of the larger one, (20 -> 30) and (30 -> 40).

    Initial angles (seeded per env): the train starts in exact conjugate mesh -- a tooth of
    one gear centred in a gap of the next on the line of centres -- turned by a common
    phase theta ~U(0, one pitch of the driver) through the gear ratios, then the two
    driven gears are each turned by an independent jitter of at most a fifth of the
    backlash (arc length on their pitch circles)."""
    rng = np.random.default_rng(seed)
    z1, z2, z3 = GEAR_TEETH
    m = module_mm * 1e-3
    assets = gear_assets(module_mm, GEAR_TEETH, 10.0, backlash_mm, tri_target, n_samples, sdf_res, rng)
    c12 = m * (z1 + z2) / 2
    c23 = m * (z2 + z3) / 2
    centres = [(0.0, 0.0, 0.0), (c12, 0.0, 0.0), (c12 + c23, 0.0, 0.0)]
    bodies = np.zeros((n_envs, 3), dtype=BODY_DTYPE)
    jit = 0.2 * backlash_mm * 1e-3
    for e in range(n_envs):
        th = rng.uniform(0.0, 2 * np.pi / z1)
        a2 = np.pi / z2 - th * z1 / z2 + rng.uniform(-jit, jit) / (m * z2 / 2)
        a3 = th * z1 / z3 + rng.uniform(-jit, jit) / (m * z3 / 2)
        z_axis = [0, 0, 1]
        bodies[e, 0] = _body(0, KINEMATIC, centres[0], quat_axis_angle(z_axis, th), mu,
                             angvel=(0, 0, drive_rate))
        bodies[e, 1] = _body(1, FIXED_AXIS, centres[1], quat_axis_angle(z_axis, a2), mu, axis=(0, 0, 1))
        bodies[e, 2] = _body(2, FIXED_AXIS, centres[2], quat_axis_angle(z_axis, a3), mu, axis=(0, 0, 1),
                             torque=(0, 0, -load_torque))
    pairs = np.array([[0, 1], [1, 2]], dtype=np.int32)
    sim = SimParams(n_substeps=n_substeps, n_iters=n_iters, frames=frames)
    return Scene("gears", assets, [EnvGroup(bodies, pairs)], sim)


# --------------------------------------------------------------------------------------
# piles of nuts: several free bodies per env, coupled through their contacts
# --------------------------------------------------------------------------------------
def _random_quat(rng: np.random.Generator) -> np.ndarray:
    """uniform random rotation (normalised Gaussian quaternion), w >= 0"""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    return q if q[3] >= 0 else -q


def pile_scene(n_envs: int = 256, seed: int = 0, n_nuts: int = 7, mode: str = "drop", n_samples: int = 5000,
               sdf_res: int = 128, mu: float = 0.3, n_substeps: int = 8, n_iters: int = 32,
               frames: int = 120, sink_mm: float = 0.02) -> Scene:
    """Piles of ISO M16 nuts (the M16 nut of nut_bolt_scene, 18,136 triangles, n_samples
    samples and its own 128^3 SDF) on a static 120 x 120 x 10 mm plate whose top face is
    z = 0.  Every nut is a free body; the pairs are nut -> plate for every nut and nut i ->
    nut j (samples of i against the SDF of j) for every i < j, so an env couples up to
    n_nuts + 1 <= 8 bodies through up to 28 pairs.

    mode "drop": the nuts start at random orientations and positions (xy within +-25 mm,
    heights 10-100 mm) with their bounding spheres 1 mm apart or more, and fall into a pile.
    mode "stacks": resting stacks of one to three nuts lying flat (random yaw, xy offsets
    of a stack's nuts within 1 mm), each nut sunk sink_mm into the one below (or the
    plate), the stacks' bounding spheres apart: contacts from the first substep."""
    if not 1 <= n_nuts <= 7:
        raise ValueError("n_nuts must be 1..7 (8 bodies per env at most)")
    rng = np.random.default_rng(seed)
    P, af, _ = ISO_COARSE[16]
    thick = 13.0e-3
    nV, nT = nut_mesh(16, P, 13.0, af, 0.05, n_ang=84)
    nut = Asset("nut_m16", nV, nT, sample_surface(nV, nT, n_samples, rng), 7800.0, sdf_res=sdf_res, sdf_pad=1e-3)
    PV, PT = box_mesh(0.06, 0.06, 0.005)
    plate = Asset("plate", PV, PT, None, 7800.0, sdf_res=sdf_res, sdf_pad=1e-3)
    r = float(np.linalg.norm(nV, axis=1).max())
    bodies = np.zeros((n_envs, n_nuts + 1), dtype=BODY_DTYPE)
    for e in range(n_envs):
        if mode == "drop":
            pos = []
            while len(pos) < n_nuts:
                c = np.array([rng.uniform(-0.025, 0.025), rng.uniform(-0.025, 0.025), rng.uniform(0.010, 0.100)])
                if c[2] - r < 0.0005:
                    continue
                if all(np.linalg.norm(c - o) >= 2 * r + 1e-3 for o in pos):
                    pos.append(c)
            for k, c in enumerate(pos):
                bodies[e, k] = _body(0, DYNAMIC, tuple(c), _random_quat(rng), mu)
        elif mode == "stacks":
            heights = []
            while sum(heights) < n_nuts:
                heights.append(int(rng.integers(1, min(3, n_nuts - sum(heights)) + 1)))
            centres = []
            while len(centres) < len(heights):
                c = rng.uniform(-0.045, 0.045, 2)
                if all(np.linalg.norm(c - o) >= 2 * r + 1e-3 for o in centres):
                    centres.append(c)
            k = 0
            for c, hgt in zip(centres, heights):
                for level in range(hgt):
                    z = thick / 2 + level * thick - (level + 1) * sink_mm * 1e-3
                    xy = c + rng.uniform(-1e-3, 1e-3, 2)
                    bodies[e, k] = _body(0, DYNAMIC, (xy[0], xy[1], z),
                                         quat_axis_angle([0, 0, 1], rng.uniform(0, np.pi / 3)), mu)
                    k += 1
        else:
            raise ValueError(f"unknown pile mode {mode!r}")
        bodies[e, n_nuts] = _body(1, STATIC, (0.0, 0.0, -0.005), (0, 0, 0, 1), mu)
    pairs = [(k, n_nuts) for k in range(n_nuts)] + [(i, j) for i in range(n_nuts) for j in range(i + 1, n_nuts)]
    sim = SimParams(n_substeps=n_substeps, n_iters=n_iters, frames=frames)
    return Scene("pile", [nut, plate], [EnvGroup(bodies, np.array(pairs, np.int32))], sim)


# --------------------------------------------------------------------------------------
# one env of hundreds of nuts (pile env): the pairs are found at every detection
# --------------------------------------------------------------------------------------
# the paper's three pile bodies (Sec. III-D scene list; Table "geometric representations":
# the torus's SDF box is 304 x 104 x 304 voxels, (R + r) / r = 2.92; the bowl's 257 x 75 x
# 257, rim diameter / depth = 3.43, with 582 vertices)
PILE_BODIES = ("nut", "torus", "bowl")


def pile_body_asset(kind: str, n_samples: int, sdf_res: int, rng: np.random.Generator):
    """(asset, stack step, rest height of the body's origin above its support): an M16 nut
    (24 AF x 13 mm, 18,136 triangles); a torus R = 15.4 mm, r = 8 mm (64 x 16 segments,
    2,048 triangles); a bowl of rim diameter 100 mm, depth 29 mm, wall 2 mm (578 vertices,
    1,152 triangles), which nests in the bowl below it."""
    if kind == "nut":
        P, af, _ = ISO_COARSE[16]
        V, T = nut_mesh(16, P, 13.0, af, 0.05, n_ang=84)
        step, rest = 13.0e-3, 6.5e-3
    elif kind == "torus":
        V, T = torus_mesh(15.4e-3, 8.0e-3, 64, 16)
        step, rest = 16.0e-3, 8.0e-3
    elif kind == "bowl":
        V, T = bowl_mesh(50.0e-3, 29.0e-3, 2.0e-3)
        step, rest = 2.0e-3, 0.0
    else:
        raise ValueError(f"unknown pile body {kind!r}")
    a = Asset(f"{kind}_pile", V, T, sample_surface(V, T, n_samples, rng), 7800.0 if kind == "nut" else 2500.0,
              sdf_res=sdf_res, sdf_pad=1e-3)
    return a, step, rest


def pile_env_scene(kind: str = "nut", n_bodies: int = 1023, seed: int = 0, mode: str = "drop",
                   n_samples: int = 5000, sdf_res: int = 128, plate_sdf_res: int = 128, mu: float = 0.3,
                   n_substeps: int = 4, n_iters: int = 16, n_vel_iters: int = 1, frames: int = 120,
                   gap_mm: float = 2.0, layers: int = 4, sink_mm: float = 0.02, overlap_mm: float = 1.0) -> Scene:
    """The paper's pile scenes: n_bodies nuts, toruses or bowls in ONE env over a static
    support (SDF only, no samples; its floor at z = 0), as a pile env whose pairs every
    detection finds again.

    mode "drop": the bodies start in a square lattice of columns (`layers` deep, cells of
    the body's bounding diameter plus gap_mm, jittered by up to a quarter of the gap), at
    random orientations, the lowest layer gap_mm above the floor, and fall into a pile
    inside a round tray (a box with a blind cylindrical hole 60 mm deep, a floor of 15 mm or
    four tray voxels below it, the hole's wall 10 mm outside the lattice's corners) that
    keeps every body on the floor.
    mode "heap": resting stacks of one to three bodies lying flat (random yaw), each sunk
    sink_mm into the one below or the floor (bowls nest in the bowl below); the stacks
    stand on a square grid whose pitch is the body's largest radius in the xy plane times
    two less overlap_mm, so that neighbouring stacks touch where their outlines meet."""
    if not 1 <= n_bodies <= 1023:
        raise ValueError("n_bodies must be 1..1023 (a pile env holds 1024 bodies with the support)")
    rng = np.random.default_rng(seed)
    body, step, rest = pile_body_asset(kind, n_samples, sdf_res, rng)
    V = body.verts
    r = float(np.linalg.norm(V, axis=1).max())              # bounding sphere (about the origin)
    rc = float(np.linalg.norm(V[:, :2], axis=1).max())      # largest radius in the xy plane
    bodies = np.zeros(n_bodies + 1, dtype=BODY_DTYPE)
    if mode == "drop":
        cell = 2 * r + gap_mm * 1e-3
        m = max(1, int(math.ceil(math.sqrt(n_bodies / layers))))
        for k in range(n_bodies):
            lay, rem = divmod(k, m * m)
            iy, ix = divmod(rem, m)
            jit = rng.uniform(-0.25, 0.25, 2) * gap_mm * 1e-3
            # the bounding sphere of a body is centred on its origin for the nut and the torus
            # and reaches below it for the bowl: keep the sphere gap_mm above the floor
            c = ((ix - (m - 1) / 2) * cell + jit[0], (iy - (m - 1) / 2) * cell + jit[1],
                 r + gap_mm * 1e-3 + lay * cell)
            bodies[k] = _body(0, DYNAMIC, c, _random_quat(rng), mu)
        R = math.sqrt(2.0) * m * cell / 2 + 0.01
        # the floor below the hole is at least 15 mm and four of the tray's voxels thick
        floor = max(0.015, 4.0 * (2 * R + 0.04) / plate_sdf_res)
        TV, TT = box_with_hole_mesh(2 * R + 0.04, 2 * R + 0.04, 0.06 + floor, R, 0.06, 64)
        support = Asset("tray", TV, TT, None, 7800.0, sdf_res=plate_sdf_res, sdf_pad=1e-3)
        support_z = 0.06
    elif mode == "heap":
        pitch = 2 * rc - overlap_mm * 1e-3
        heights = []
        while sum(heights) < n_bodies:
            heights.append(int(rng.integers(1, min(3, n_bodies - sum(heights)) + 1)))
        m = max(1, int(math.ceil(math.sqrt(len(heights)))))
        k = 0
        for si, hgt in enumerate(heights):
            iy, ix = divmod(si, m)
            cx, cy = (ix - (m - 1) / 2) * pitch, (iy - (m - 1) / 2) * pitch
            for level in range(hgt):
                z = rest + level * step - (level + 1) * sink_mm * 1e-3
                bodies[k] = _body(0, DYNAMIC, (cx, cy, z), quat_axis_angle([0, 0, 1], rng.uniform(0, np.pi / 3)), mu)
                k += 1
        half = m * pitch / 2 + 0.02
        PV, PT = box_mesh(half, half, 0.005)
        support = Asset("plate", PV, PT, None, 7800.0, sdf_res=plate_sdf_res, sdf_pad=1e-3)
        support_z = -0.005
    else:
        raise ValueError(f"unknown pile mode {mode!r}")
    bodies[n_bodies] = _body(1, STATIC, (0.0, 0.0, support_z), (0, 0, 0, 1), mu)
    sim = SimParams(n_substeps=n_substeps, n_iters=n_iters, n_vel_iters=n_vel_iters, frames=frames)
    return Scene(f"{kind}_pile_env", [body, support], [], sim, piles=[bodies])


def nut_pile_env_scene(n_nuts: int = 1024, seed: int = 0, mode: str = "drop", n_samples: int = 5000,
                       sdf_res: int = 128, plate_sdf_res: int = 128, mu: float = 0.3, n_substeps: int = 4,
                       n_iters: int = 16, n_vel_iters: int = 1, frames: int = 120, gap_mm: float = 2.0,
                       layers: int = 4, sink_mm: float = 0.02, overlap_mm: float = 1.0) -> Scene:
    """The paper's Nuts scene: pile_env_scene of ISO M16 nuts (the nut of nut_bolt_scene,
    its own SDF, n_samples samples).  In mode "heap" the grid pitch is the nut's
    across-corners width less overlap_mm, so that hexagon corners of neighbouring stacks
    touch: nut-plate, nut-on-nut and side contacts from the first substep."""
    return pile_env_scene("nut", n_nuts, seed=seed, mode=mode, n_samples=n_samples, sdf_res=sdf_res,
                          plate_sdf_res=plate_sdf_res, mu=mu, n_substeps=n_substeps, n_iters=n_iters,
                          n_vel_iters=n_vel_iters, frames=frames, gap_mm=gap_mm, layers=layers, sink_mm=sink_mm,
                          overlap_mm=overlap_mm)
