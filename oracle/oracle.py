"""ctypes wrapper of the FP64 CPU oracle (fw_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only tests/, the package's smoke check and bench.py's
CPU-baseline leg may import this module.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fw_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (-O2, OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "fw_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-fPIC",
                               "-shared", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrConfig(C.Structure):
    _fields_ = [("gravity", C.c_double * 3), ("dt", C.c_double), ("contact_offset", C.c_double),
                ("cos_patch", C.c_double), ("max_patches", C.c_int), ("batch_size", C.c_int),
                ("baumgarte", C.c_double), ("n_vel_iters", C.c_int), ("max_angvel", C.c_double),
                ("margin_len", C.c_double), ("margin_dot", C.c_double), ("n_threads", C.c_int),
                ("contact_gen", C.c_int), ("tri_iters", C.c_int), ("sdf_band", C.c_float),
                ("solver", C.c_int)]


CONTACT_DTYPE = np.dtype([("sample", np.int32), ("patch", np.int32), ("phi", np.float64),
                          ("xa", np.float64, 3), ("xb", np.float64, 3), ("n", np.float64, 3)],
                         align=True)
CANDIDATE_DTYPE = np.dtype([("sample", np.int32), ("phi", np.float32), ("x", np.float32, 3),
                            ("n", np.float32, 3)])

_P = np.ctypeslib.ndpointer
_f32 = _P(dtype=np.float32, flags="C_CONTIGUOUS")
_f64 = _P(dtype=np.float64, flags="C_CONTIGUOUS")
_i32 = _P(dtype=np.int32, flags="C_CONTIGUOUS")
_u8 = _P(dtype=np.uint8, flags="C_CONTIGUOUS")
_i64 = _P(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp = C.c_void_p
            L.or_closest_point_triangle.argtypes = [_f64, _f64, _f64, _f64, _f64]
            L.or_closest_point_triangle.restype = C.c_int
            L.or_solid_angle.argtypes = [_f64, _f64, _f64, _f64]
            L.or_solid_angle.restype = C.c_double
            L.or_winding_number.argtypes = [_f64, _f32, _i32, C.c_int]
            L.or_winding_number.restype = C.c_double
            L.or_point_mesh_distance.argtypes = [_f64, _f32, _i32, C.c_int]
            L.or_point_mesh_distance.restype = C.c_double
            L.or_mass_properties.argtypes = [_f32, _i32, C.c_int, C.c_double, C.POINTER(C.c_double),
                                             _f64, _f64]
            L.or_grid_params.argtypes = [_f32, C.c_int, C.c_int, C.c_float, C.c_int, _f32,
                                         C.POINTER(C.c_float), _i32]
            L.or_bake_nodes.argtypes = [_f32, _i32, C.c_int, _f32, C.c_float, _i32, vp,
                                        C.c_longlong, _f64, C.c_int]
            L.or_query.argtypes = [_f64, _f32, C.c_float, _i32, _f32, C.c_int, _f64, _f64, _i32]
            L.or_query_band.argtypes = [_f64, _f32, C.c_float, _i32, C.c_float, _f32, C.c_int, _f64, _f64, _i32,
                                        C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.or_create.argtypes = [C.POINTER(OrConfig)]
            L.or_create.restype = vp
            L.or_destroy.argtypes = [vp]
            L.or_set_threads.argtypes = [vp, C.c_int]
            L.or_add_asset.argtypes = [vp, _f32, C.c_int, _i32, C.c_int, vp, C.c_int, C.c_double]
            L.or_asset_bake.argtypes = [vp, C.c_int, C.c_int, C.c_float, C.c_int, C.c_int]
            L.or_asset_set_grid.argtypes = [vp, C.c_int, _f32, C.c_float, _i32, _f32]
            L.or_asset_get_grid.argtypes = [vp, C.c_int, _f32, C.POINTER(C.c_float), _i32]
            L.or_asset_mass.argtypes = [vp, C.c_int, C.POINTER(C.c_double), _f64, _f64]
            L.or_add_envs.argtypes = [vp, C.c_int, vp, C.c_int, _i32, C.c_int]
            L.or_get_pile_pairs.argtypes = [vp, C.c_int, _i32, _i32, C.c_int, C.POINTER(C.c_int)]
            L.or_pair_margins.argtypes = [vp, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_find_pile_pairs.argtypes = [vp, C.c_int]
            L.or_n_envs.argtypes = [vp]
            L.or_n_bodies.argtypes = [vp]
            L.or_step.argtypes = [vp, C.c_int, C.c_int]
            L.or_substep.argtypes = [vp, C.c_double, C.c_int, C.c_int]
            L.or_collide.argtypes = [vp]
            L.or_get_contacts.argtypes = [vp, C.c_int, vp, C.c_int, C.POINTER(C.c_int),
                                          C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_set_contacts.argtypes = [vp, C.c_int, vp, C.c_int]
            L.or_get_pair_contacts.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, C.POINTER(C.c_int)]
            L.or_set_pair_contacts.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int]
            L.or_env_margins.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_reset_margins.argtypes = [vp]
            L.or_get_state.argtypes = [vp, _f64, _f64, _f64, _f64]
            L.or_set_state.argtypes = [vp, _f64, _f64, _f64, _f64]
            L.or_get_impulses.argtypes = [vp, C.c_int, _f64, C.c_int, C.POINTER(C.c_int)]
            L.or_bake_seconds.argtypes = [vp]
            L.or_bake_seconds.restype = C.c_double
            L.or_query_pair.argtypes = [vp, C.c_int, C.c_int, _f64, _f64, _i32, _f64]
            L.or_pair_candidates.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int, C.POINTER(C.c_int)]
            L.or_tri_contacts.argtypes = [vp, C.c_int, C.c_int, _f64, _f64, _f64, _i32, _f64]
            L.or_diff_record.argtypes = [vp, C.c_int, C.c_int]
            L.or_diff_replay.argtypes = [vp]
            L.or_diff_adjoint.argtypes = [vp] + [_f64] * 10
            L.or_diff_tape_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                            C.POINTER(C.c_double), C.POINTER(C.c_int)]
            L.or_diff_get_tape.argtypes = [vp, _i32, _i32, _u8, _u8]
            L.or_diff_set_tape.argtypes = [vp, C.c_int, C.c_int, C.c_double, _i32, _i32, _u8, _u8]
            L.or_set_body_mass.argtypes = [vp, C.c_int, C.c_double]
            L.or_set_pair_mu.argtypes = [vp, C.c_int, C.c_double]
            L.or_n_pairs.argtypes = [vp]
            L.or_get_body_mass.argtypes = [vp, C.c_int]
            L.or_get_body_mass.restype = C.c_double
            L.or_get_pair_mu.argtypes = [vp, C.c_int]
            L.or_get_pair_mu.restype = C.c_double
            L.or_reduce.argtypes = [vp, C.c_int, C.c_double, C.c_int, C.c_int, vp, C.c_int,
                                    C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]
            _lib = L
    return _lib


def _d3(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(3))


# ---- primitives -------------------------------------------------------------------------
def closest_point_triangle(p, a, b, c) -> Tuple[np.ndarray, int]:
    q = np.zeros(3)
    r = lib().or_closest_point_triangle(_d3(p), _d3(a), _d3(b), _d3(c), q)
    return q, r


def solid_angle(p, a, b, c) -> float:
    return lib().or_solid_angle(_d3(p), _d3(a), _d3(b), _d3(c))


def _mesh(V, T):
    return (np.ascontiguousarray(V, dtype=np.float32), np.ascontiguousarray(T, dtype=np.int32))


def winding_number(p, V, T) -> float:
    V, T = _mesh(V, T)
    return lib().or_winding_number(_d3(p), V, T, len(T))


def point_mesh_distance(p, V, T) -> float:
    V, T = _mesh(V, T)
    return lib().or_point_mesh_distance(_d3(p), V, T, len(T))


def mass_properties(V, T, density: float):
    V, T = _mesh(V, T)
    m = C.c_double()
    com, I = np.zeros(3), np.zeros(9)
    lib().or_mass_properties(V, T, len(T), density, C.byref(m), com, I)
    return m.value, com, I.reshape(3, 3)


def grid_params(V, res: int, pad: float, cubic: bool = True):
    V = np.ascontiguousarray(V, dtype=np.float32)
    lo, dims, h = np.zeros(3, np.float32), np.zeros(3, np.int32), C.c_float()
    lib().or_grid_params(V, len(V), res, pad, int(cubic), lo, C.byref(h), dims)
    return lo, np.float32(h.value), dims


def bake_nodes(V, T, lo, h, dims, nodes: Optional[np.ndarray] = None, n_threads: int = 0):
    V, T = _mesh(V, T)
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    if nodes is None:
        out = np.zeros(int(np.prod(dims.astype(np.int64))))
        lib().or_bake_nodes(V, T, len(T), lo, h, dims, None, 0, out, n_threads)
        return out.reshape(dims[2], dims[1], dims[0])
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.zeros(len(nodes))
    lib().or_bake_nodes(V, T, len(T), lo, h, dims, nodes.ctypes.data, len(nodes), out, n_threads)
    return out


def query(grid: np.ndarray, lo, h, dims, pts):
    g = np.ascontiguousarray(grid, dtype=np.float64).reshape(-1)
    pts = np.ascontiguousarray(pts, dtype=np.float32).reshape(-1, 3)
    n = len(pts)
    phi, grad, valid = np.zeros(n), np.zeros((n, 3)), np.zeros(n, np.int32)
    lib().or_query(g, np.ascontiguousarray(lo, np.float32), h, np.ascontiguousarray(dims, np.int32),
                   pts, n, phi, grad, valid)
    return phi, grad, valid.astype(bool)


def query_band(grid: np.ndarray, lo, h, dims, band_voxels: float, pts):
    """query() with the grid held in narrow-band bricks (R17): (phi, grad, valid, bricks
    stored, bricks in all)."""
    g = np.ascontiguousarray(grid, dtype=np.float64).reshape(-1)
    pts = np.ascontiguousarray(pts, dtype=np.float32).reshape(-1, 3)
    n = len(pts)
    phi, grad, valid = np.zeros(n), np.zeros((n, 3)), np.zeros(n, np.int32)
    ns, nb = C.c_int(), C.c_int()
    lib().or_query_band(g, np.ascontiguousarray(lo, np.float32), h, np.ascontiguousarray(dims, np.int32),
                        band_voxels, pts, n, phi, grad, valid, C.byref(ns), C.byref(nb))
    return phi, grad, valid.astype(bool), ns.value, nb.value


def reduce(cands: np.ndarray, cos_patch: float = 0.94, max_patches: int = 128,
           batch_size: int = 1024):
    """Algorithm 1 on a CANDIDATE_DTYPE array -> (contacts, n_patches, margin_len, margin_dot)."""
    cands = np.ascontiguousarray(cands, dtype=CANDIDATE_DTYPE)
    cap = max(7 * max_patches, 1)
    out = np.zeros(cap, CONTACT_DTYPE)
    n, npch, ml, md = C.c_int(), C.c_int(), C.c_double(), C.c_double()
    lib().or_reduce(cands.ctypes.data, len(cands), cos_patch, max_patches, batch_size,
                    out.ctypes.data, cap, C.byref(n), C.byref(npch), C.byref(ml), C.byref(md))
    return out[: n.value].copy(), npch.value, ml.value, md.value


# ---- world ------------------------------------------------------------------------------
class OracleWorld:
    """The oracle's world, built from a scenes.Scene (or by hand)."""

    def __init__(self, sim=None, n_threads: int = 0, margin_len: float = 1e-7,
                 margin_dot: float = 1e-6, **over):
        cfg = OrConfig()
        g = getattr(sim, "gravity", (0.0, 0.0, -9.81))
        cfg.gravity[:] = list(over.get("gravity", g))
        cfg.dt = over.get("dt", getattr(sim, "dt", 1.0 / 60.0))
        cfg.contact_offset = over.get("contact_offset", getattr(sim, "contact_offset", 1e-4))
        cfg.cos_patch = over.get("cos_patch", getattr(sim, "cos_patch", 0.94))
        cfg.max_patches = over.get("max_patches", getattr(sim, "max_patches", 128))
        cfg.batch_size = over.get("batch_size", getattr(sim, "batch_size", 1024))
        cfg.baumgarte = over.get("baumgarte", getattr(sim, "baumgarte", 0.2))
        cfg.n_vel_iters = over.get("n_vel_iters", getattr(sim, "n_vel_iters", 0))
        cfg.max_angvel = over.get("max_angvel", getattr(sim, "max_angvel", 0.0))
        cfg.contact_gen = over.get("contact_gen", 0)
        cfg.tri_iters = over.get("tri_iters", 16)
        cfg.sdf_band = over.get("sdf_band", 0.0)
        cfg.solver = over.get("solver", 0)
        cfg.margin_len = margin_len
        cfg.margin_dot = margin_dot
        cfg.n_threads = n_threads
        self.cfg = cfg
        self.h = lib().or_create(C.byref(cfg))
        self.n_assets = 0

    def set_threads(self, n_threads: int):
        """OpenMP threads for this world's later calls (0: the OpenMP default)."""
        lib().or_set_threads(self.h, n_threads)

    def close(self):
        if self.h:
            lib().or_destroy(self.h)
            self.h = None

    __del__ = close

    def add_asset(self, V, T, samples=None, density=7800.0) -> int:
        V, T = _mesh(V, T)
        if samples is not None:
            samples = np.ascontiguousarray(samples, dtype=np.float32)
            sp, ns = samples.ctypes.data, len(samples)
        else:
            sp, ns = None, 0
        self._keep = getattr(self, "_keep", []) + [samples]
        a = lib().or_add_asset(self.h, V, len(V), T, len(T), sp, ns, density)
        self.n_assets += 1
        return a

    def bake(self, asset: int, res: int, pad: float, cubic: bool = True, lazy: bool = False):
        lib().or_asset_bake(self.h, asset, res, pad, int(cubic), int(lazy))

    def set_grid(self, asset: int, lo, h, dims, values: np.ndarray):
        lib().or_asset_set_grid(self.h, asset, np.ascontiguousarray(lo, np.float32), float(h),
                                np.ascontiguousarray(dims, np.int32),
                                np.ascontiguousarray(values, np.float32).reshape(-1))

    def grid(self, asset: int):
        lo, dims, h = np.zeros(3, np.float32), np.zeros(3, np.int32), C.c_float()
        lib().or_asset_get_grid(self.h, asset, lo, C.byref(h), dims)
        return lo, np.float32(h.value), dims

    def mass(self, asset: int):
        m = C.c_double()
        com, I = np.zeros(3), np.zeros(9)
        lib().or_asset_mass(self.h, asset, C.byref(m), com, I)
        return m.value, com, I.reshape(3, 3)

    def add_envs(self, bodies: np.ndarray, pairs) -> int:
        """pairs: (n, 2) local body ids, or None for pile envs (R20: pairs found by the
        broad phase at every detection)."""
        bodies = np.ascontiguousarray(bodies)
        assert bodies.dtype.itemsize == 104
        if pairs is None:
            return lib().or_add_envs(self.h, bodies.shape[0], bodies.ctypes.data, bodies.shape[1],
                                     np.zeros(1, np.int32), -1)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1)
        return lib().or_add_envs(self.h, bodies.shape[0], bodies.ctypes.data, bodies.shape[1],
                                 pairs, len(pairs) // 2)

    def pile_pairs(self, env: int):
        """(pairs (n, 2) of local body ids (point body, SDF body), colours (n,)) of a pile
        env's last detection / solve."""
        cap = 1 << 16
        ab, col, n = np.zeros(2 * cap, np.int32), np.zeros(cap, np.int32), C.c_int()
        if lib().or_get_pile_pairs(self.h, env, ab, col, cap, C.byref(n)) != 0:
            raise ValueError("not a pile env, or too many pairs")
        return ab[: 2 * n.value].reshape(-1, 2).copy(), col[: n.value].copy()

    @property
    def n_envs(self) -> int:
        return lib().or_n_envs(self.h)

    @property
    def n_bodies(self) -> int:
        return lib().or_n_bodies(self.h)

    def step(self, n_substeps: int, n_iters: int):
        lib().or_step(self.h, n_substeps, n_iters)

    def substep(self, hs: float, n_iters: int, detect: bool = True):
        lib().or_substep(self.h, hs, n_iters, int(detect))

    def collide(self):
        lib().or_collide(self.h)

    def contacts(self, env: int):
        cap = 4096
        while True:
            out = np.zeros(cap, CONTACT_DTYPE)
            n, ml, md = C.c_int(), C.c_double(), C.c_double()
            lib().or_get_contacts(self.h, env, out.ctypes.data, cap, C.byref(n), C.byref(ml),
                                  C.byref(md))
            if n.value <= cap:
                return out[: n.value].copy(), ml.value, md.value
            cap = n.value

    def set_contacts(self, env: int, contacts: np.ndarray):
        c = np.ascontiguousarray(contacts, dtype=CONTACT_DTYPE)
        lib().or_set_contacts(self.h, env, c.ctypes.data, len(c))

    def pair_contacts(self, env: int, pair: int):
        """the contacts of one pair of the env (env-local pair index), in sweep order"""
        cap = 4096
        while True:
            out = np.zeros(cap, CONTACT_DTYPE)
            n = C.c_int()
            if lib().or_get_pair_contacts(self.h, env, pair, out.ctypes.data, cap, C.byref(n)) == 0:
                return out[: n.value].copy()
            if n.value <= cap:
                raise ValueError(f"or_get_pair_contacts: bad env {env} or pair {pair}")
            cap = n.value

    def set_pair_contacts(self, env: int, pair: int, contacts: np.ndarray):
        c = np.ascontiguousarray(contacts, dtype=CONTACT_DTYPE)
        if lib().or_set_pair_contacts(self.h, env, pair, c.ctypes.data, len(c)) != 0:
            raise ValueError(f"or_set_pair_contacts: bad env {env} or pair {pair}")

    def pair_margins(self, env: int, pair: int):
        """the smallest decision margins (length, dot) of one pair's last detection"""
        ml, md = C.c_double(), C.c_double()
        if lib().or_pair_margins(self.h, env, pair, C.byref(ml), C.byref(md)) != 0:
            raise ValueError(f"or_pair_margins: bad env {env} or pair {pair}")
        return ml.value, md.value

    def find_pile_pairs(self, env: int):
        """the pile env's pairs at the current poses (broad phase only), as pile_pairs"""
        if lib().or_find_pile_pairs(self.h, env) != 0:
            raise ValueError(f"not a pile env: {env}")
        return self.pile_pairs(env)

    def margins(self, env: int):
        ml, md = C.c_double(), C.c_double()
        lib().or_env_margins(self.h, env, C.byref(ml), C.byref(md))
        return ml.value, md.value

    def reset_margins(self):
        lib().or_reset_margins(self.h)

    def state(self):
        n = self.n_bodies
        p, q, v, w = np.zeros((n, 3)), np.zeros((n, 4)), np.zeros((n, 3)), np.zeros((n, 3))
        lib().or_get_state(self.h, p, q, v, w)
        return p, q, v, w

    def set_state(self, p, q, v, w):
        f = lambda a, k: np.ascontiguousarray(np.asarray(a, np.float64).reshape(-1, k))
        lib().or_set_state(self.h, f(p, 3), f(q, 4), f(v, 3), f(w, 3))

    def bake_seconds(self) -> float:
        return lib().or_bake_seconds(self.h)

    # ---- differentiable rollout (decisions held fixed by a tape; see fw_oracle.c)
    def diff_record(self, n_substeps: int, n_iters: int):
        if lib().or_diff_record(self.h, n_substeps, n_iters) != 0:
            raise ValueError("or_diff_record: world not differentiable")

    def diff_replay(self):
        if lib().or_diff_replay(self.h) != 0:
            raise ValueError("or_diff_replay: no tape")

    def diff_adjoint(self, g_pos, g_quat, g_lin, g_ang):
        """Adjoints of the initial state and parameters of a replay from the current state:
        dict(pos, quat, linvel, angvel (n_bodies x k), mass (n_bodies), mu (n_pairs))."""
        n, npair = self.n_bodies, lib().or_n_pairs(self.h)
        f = lambda a, k: np.ascontiguousarray(np.asarray(a, np.float64).reshape(n, k))
        out = dict(pos=np.zeros((n, 3)), quat=np.zeros((n, 4)), linvel=np.zeros((n, 3)),
                   angvel=np.zeros((n, 3)), mass=np.zeros(n), mu=np.zeros(npair))
        st = lib().or_diff_adjoint(self.h, f(g_pos, 3), f(g_quat, 4), f(g_lin, 3), f(g_ang, 3), out["pos"],
                                   out["quat"], out["linvel"], out["angvel"], out["mass"], out["mu"])
        if st != 0:
            raise ValueError("or_diff_adjoint: no tape")
        return out

    def get_tape(self):
        S, E, K, n = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        hs = C.c_double()
        if lib().or_diff_tape_info(self.h, C.byref(S), C.byref(E), C.byref(K), C.byref(hs), C.byref(n)) != 0:
            raise ValueError("no tape")
        t = dict(S=S.value, K=K.value, hs=hs.value, c_off=np.zeros(S.value * E.value + 1, np.int32),
                 c_rec=np.zeros((max(n.value, 1), 6), np.int32), r_bits=np.zeros(max(K.value * n.value, 1), np.uint8),
                 b_bits=np.zeros(S.value * E.value + 1, np.uint8))
        lib().or_diff_get_tape(self.h, t["c_off"], t["c_rec"].reshape(-1), t["r_bits"], t["b_bits"])
        t["c_rec"], t["r_bits"] = t["c_rec"][: n.value], t["r_bits"][: K.value * n.value]
        return t

    def set_tape(self, t):
        st = lib().or_diff_set_tape(self.h, int(t["S"]), int(t["K"]), float(t["hs"]),
                                    np.ascontiguousarray(t["c_off"], np.int32),
                                    np.ascontiguousarray(np.asarray(t["c_rec"], np.int32).reshape(-1)),
                                    np.ascontiguousarray(t["r_bits"], np.uint8),
                                    np.ascontiguousarray(t["b_bits"], np.uint8))
        if st != 0:
            raise ValueError("or_diff_set_tape refused the tape")

    def set_body_mass(self, body: int, mass: float):
        if lib().or_set_body_mass(self.h, body, float(mass)) != 0:
            raise ValueError("bad body or mass")

    def body_mass(self, body: int) -> float:
        return lib().or_get_body_mass(self.h, body)

    def pair_mu(self, pair: int) -> float:
        return lib().or_get_pair_mu(self.h, pair)

    def set_pair_mu(self, pair: int, mu: float):
        if lib().or_set_pair_mu(self.h, pair, float(mu)) != 0:
            raise ValueError("bad pair or mu")

    def query_pair(self, env: int, pair: int, n_samples: int):
        phi, nrm, valid = np.zeros(n_samples), np.zeros((n_samples, 3)), np.zeros(n_samples, np.int32)
        gn = np.zeros(n_samples)
        lib().or_query_pair(self.h, env, pair, phi, nrm, valid, gn)
        self.last_gnorm = gn
        return phi, nrm, valid.astype(bool)

    def tri_contacts(self, env: int, pair: int, n_tris: int):
        """Per triangle of the point body's mesh (R15): minimiser (world), phi, world normal,
        valid, and the smallest phi gap among the descent's accept/reject decisions."""
        x, n = np.zeros((n_tris, 3)), np.zeros((n_tris, 3))
        phi, margin = np.zeros(n_tris), np.zeros(n_tris)
        valid = np.zeros(n_tris, np.int32)
        lib().or_tri_contacts(self.h, env, pair, x, phi, n, valid, margin)
        return x, phi, n, valid.astype(bool), margin

    def pair_candidates(self, env: int, pair: int, cap: int = 1 << 20) -> np.ndarray:
        out = np.zeros(cap, CANDIDATE_DTYPE)
        n = C.c_int()
        lib().or_pair_candidates(self.h, env, pair, out.ctypes.data, cap, C.byref(n))
        return out[: min(n.value, cap)].copy()

    def impulses(self, env: int) -> np.ndarray:
        cap = 8192
        out = np.zeros((cap, 3))
        n = C.c_int()
        lib().or_get_impulses(self.h, env, out, cap, C.byref(n))
        return out[: min(n.value, cap)].copy()


def world_from_scene(scene, n_threads: int = 0, lazy_bake: bool = False, **over) -> OracleWorld:
    """Builds the oracle world from a scenes.Scene: assets, SDF bakes, env groups."""
    w = OracleWorld(scene.sim, n_threads=n_threads, **over)
    for a in scene.assets:
        i = w.add_asset(a.verts, a.tris, a.samples, a.density)
        if a.sdf_res:
            w.bake(i, a.sdf_res, a.sdf_pad, True, lazy_bake)
    for g in scene.groups:
        w.add_envs(g.bodies, g.pairs)
    for pb in scene.piles:
        w.add_envs(pb[None, :], None)
    return w
