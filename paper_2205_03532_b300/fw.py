"""Python binding of libfw's C ABI (include/fw.h): argument marshalling only.

Every computation happens in libfw.so; this module converts numpy arrays / torch CUDA
tensors to pointers and status codes to exceptions.  There is no fallback: if the
library is missing, creating a World fails.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Tuple

import numpy as np

from . import scenes

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfw.so")

STATUS = {0: "FW_OK", -1: "FW_ERR_ARG", -2: "FW_ERR_OOM", -3: "FW_ERR_CUDA", -4: "FW_ERR_STATE",
          -5: "FW_ERR_NONFINITE", -6: "FW_ERR_OVERFLOW", -7: "FW_ERR_TIMEOUT",
          -8: "FW_ERR_DEVICE_BOUNDS"}

# every function include/fw.h declares
ABI_FUNCTIONS = ["fw_config_default", "fw_create", "fw_destroy", "fw_add_mesh_asset", "fw_bake_sdf",
                 "fw_set_sdf", "fw_get_sdf", "fw_get_sdf_storage", "fw_get_mass", "fw_add_env_bodies", "fw_step",
                 "fw_substep", "fw_collide", "fw_get_contacts", "fw_set_contacts", "fw_get_state",
                 "fw_set_state", "fw_query_sdf", "fw_query_pair", "fw_tri_contacts", "fw_reduce", "fw_reduce_noalloc", "fw_sync",
                 "fw_set_timing", "fw_get_timings", "fw_set_solve_shape", "fw_autotune_solve", "fw_get_solve_shape",
                 "fw_record_rollout", "fw_replay_rollout", "fw_adjoint_rollout", "fw_step_fwd_ckpt",
                 "fw_step_bwd", "fw_get_tape",
                 "fw_set_body_params", "fw_get_detect_stats", "fw_get_counts", "fw_get_env_info", "fw_add_pile",
                 "fw_get_pile_pairs", "fw_set_detect_shape", "fw_set_query_cull", "fw_get_query_cull", "fw_get_detect_shape", "fw_autotune_detect",
                 "fw_test_stall",
                 "fw_launches_per_step",
                 "fw_last_error", "fw_measure_l2_read"]


class FwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class FwConfig(C.Structure):
    _fields_ = [("gravity", C.c_float * 3), ("dt", C.c_float), ("contact_offset", C.c_float),
                ("cos_patch", C.c_float), ("max_patches", C.c_int), ("patch_dirs", C.c_int),
                ("batch_size", C.c_int),
                ("baumgarte", C.c_float), ("n_vel_iters", C.c_int), ("max_angvel", C.c_float),
                ("sdf_fp16", C.c_int), ("contact_gen", C.c_int), ("tri_iters", C.c_int), ("sdf_band", C.c_float),
                ("solver", C.c_int), ("device", C.c_int),
                ("cuda_stream", C.c_void_p), ("seed", C.c_ulonglong)]


CONTACT_DTYPE = np.dtype([("sample", np.int32), ("patch", np.int32), ("pair", np.int32),
                          ("phi", np.float32), ("xa", np.float32, 3), ("xb", np.float32, 3),
                          ("n", np.float32, 3)])
CANDIDATE_DTYPE = np.dtype([("sample", np.int32), ("phi", np.float32), ("x", np.float32, 3),
                            ("n", np.float32, 3)])
assert CONTACT_DTYPE.itemsize == 52 and CANDIDATE_DTYPE.itemsize == 32
assert scenes.BODY_DTYPE.itemsize == 104

_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libfw.so and declares the ABI's signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"libfw.so not built at {path}; run paper_2205_03532_b300.csrc.build")
    L = C.CDLL(path)
    vp, i, f, st = C.c_void_p, C.c_int, C.c_float, C.c_int
    sig = {
        "fw_config_default": (None, [C.POINTER(FwConfig)]),
        "fw_create": (st, [C.POINTER(FwConfig), C.POINTER(vp)]),
        "fw_destroy": (st, [vp]),
        "fw_add_mesh_asset": (st, [vp, vp, i, vp, i, vp, i, f, C.POINTER(i)]),
        "fw_bake_sdf": (st, [vp, i, i, f, i]),
        "fw_set_sdf": (st, [vp, i, vp, f, vp, vp]),
        "fw_get_sdf": (st, [vp, i, vp, C.POINTER(f), vp, vp]),
        "fw_get_mass": (st, [vp, i, vp, vp, vp]),
        "fw_get_sdf_storage": (st, [vp, i, C.POINTER(C.c_longlong), C.POINTER(i), C.POINTER(i)]),
        "fw_add_env_bodies": (st, [vp, i, vp, i, vp, i, C.POINTER(i)]),
        "fw_add_pile": (st, [vp, vp, i, i, i, C.POINTER(i)]),
        "fw_get_pile_pairs": (st, [vp, i, vp, vp, i, C.POINTER(i)]),
        "fw_set_detect_shape": (st, [vp, i, i]),
        "fw_set_query_cull": (st, [vp, i]),
        "fw_get_query_cull": (st, [vp, C.POINTER(i)]),
        "fw_test_stall": (st, [vp, i]),
        "fw_get_detect_shape": (st, [vp, C.POINTER(i), C.POINTER(i)]),
        "fw_autotune_detect": (st, [vp, i, C.POINTER(i), C.POINTER(i), C.POINTER(C.c_float)]),
        "fw_step": (st, [vp, i, i]),
        "fw_substep": (st, [vp, f, i, i]),
        "fw_collide": (st, [vp]),
        "fw_get_contacts": (st, [vp, i, vp, i, C.POINTER(i)]),
        "fw_set_contacts": (st, [vp, i, vp, i]),
        "fw_get_state": (st, [vp, vp, vp, vp, vp, i]),
        "fw_set_state": (st, [vp, vp, vp, vp, vp, i]),
        "fw_query_sdf": (st, [vp, i, vp, i, vp, vp, i]),
        "fw_query_pair": (st, [vp, i, i, vp, vp, i]),
        "fw_tri_contacts": (st, [vp, i, i, vp, vp, vp, i]),
        "fw_reduce": (st, [vp, vp, i, vp, i, C.POINTER(i), C.POINTER(i)]),
        "fw_reduce_noalloc": (st, [vp, vp, i, vp, i, vp]),
        "fw_sync": (st, [vp]),
        "fw_set_timing": (st, [vp, i]),
        "fw_get_timings": (st, [vp, vp, i]),
        "fw_set_solve_shape": (st, [vp, i, i]),
        "fw_get_solve_shape": (st, [vp, C.POINTER(i), C.POINTER(i)]),
        "fw_autotune_solve": (st, [vp, i, i, i, C.POINTER(i), C.POINTER(i), C.POINTER(C.c_float)]),
        "fw_record_rollout": (st, [vp, i, i]),
        "fw_replay_rollout": (st, [vp]),
        "fw_adjoint_rollout": (st, [vp] + [vp] * 10 + [i]),
        "fw_step_fwd_ckpt": (st, [vp, i, i]),
        "fw_step_bwd": (st, [vp] + [vp] * 10 + [i]),
        "fw_get_tape": (st, [vp, vp, vp, vp, vp, vp]),
        "fw_set_body_params": (st, [vp, vp, vp]),
        "fw_get_detect_stats": (st, [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "fw_get_counts": (st, [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i)]),
        "fw_get_env_info": (st, [vp, i, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i)]),
        "fw_launches_per_step": (i, [vp, i]),
        "fw_last_error": (C.c_char_p, [vp]),
        "fw_measure_l2_read": (st, [i, C.c_longlong, i, C.POINTER(f)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def measure_l2_read(device: int = 0, nbytes: int = 48 << 20, iters: int = 200) -> float:
    """L2 read bandwidth of a device in GB/s (fw_measure_l2_read)."""
    L = load_library()
    g = C.c_float(0.0)
    st = L.fw_measure_l2_read(device, nbytes, iters, C.byref(g))
    if st != 0:
        raise FwError(st, "fw_measure_l2_read failed")
    return float(g.value)


def default_config(**over) -> FwConfig:
    cfg = FwConfig()
    load_library().fw_config_default(C.byref(cfg))
    for k, v in over.items():
        if k == "gravity":
            cfg.gravity[:] = list(v)
        else:
            setattr(cfg, k, v)
    return cfg


def _ptr(a):
    """(pointer, is_device) of a numpy array or a torch tensor."""
    if a is None:
        return None, False
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), bool(a.is_cuda)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, False


class World:
    """One libfw world.  Methods map one to one to the ABI calls."""

    def __init__(self, cfg: Optional[FwConfig] = None, **over):
        self.lib = load_library()
        self.cfg = cfg if cfg is not None else default_config(**over)
        h = C.c_void_p()
        st = self.lib.fw_create(C.byref(self.cfg), C.byref(h))
        if st != 0:
            raise FwError(st, "fw_create failed")
        self.h = h

    def _check(self, status):
        if status != 0:
            msg = self.lib.fw_last_error(self.h) or b""
            raise FwError(status, msg.decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.fw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- assets
    def add_mesh_asset(self, verts, tris, samples=None, density=7800.0) -> int:
        V = np.ascontiguousarray(verts, np.float32)
        T = np.ascontiguousarray(tris, np.int32)
        S = None if samples is None else np.ascontiguousarray(samples, np.float32)
        out = C.c_int()
        self._check(self.lib.fw_add_mesh_asset(self.h, V.ctypes.data, len(V), T.ctypes.data, len(T),
                                               None if S is None else S.ctypes.data,
                                               0 if S is None else len(S), density, C.byref(out)))
        return out.value

    def bake_sdf(self, asset: int, resolution: int, padding: float = 1e-3, cubic: bool = True):
        self._check(self.lib.fw_bake_sdf(self.h, asset, resolution, padding, int(cubic)))

    def set_sdf(self, asset: int, lo, h: float, dims, values):
        lo = np.ascontiguousarray(lo, np.float32)
        dims = np.ascontiguousarray(dims, np.int32)
        v = np.ascontiguousarray(values, np.float32)
        self._check(self.lib.fw_set_sdf(self.h, asset, lo.ctypes.data, float(h), dims.ctypes.data, v.ctypes.data))

    def get_sdf(self, asset: int, values: bool = True):
        lo, dims, h = np.zeros(3, np.float32), np.zeros(3, np.int32), C.c_float()
        self._check(self.lib.fw_get_sdf(self.h, asset, lo.ctypes.data, C.byref(h), dims.ctypes.data, None))
        vals = None
        if values:
            vals = np.zeros((dims[2], dims[1], dims[0]), np.float32)
            self._check(self.lib.fw_get_sdf(self.h, asset, None, None, None, vals.ctypes.data))
        return lo, np.float32(h.value), dims, vals

    def sdf_storage(self, asset: int):
        """(bytes of the SDF lookup copy, bricks kept, bricks in all) (fw_get_sdf_storage;
        the brick counts are 0 for dense storage)"""
        b, ns, nb = C.c_longlong(), C.c_int(), C.c_int()
        self._check(self.lib.fw_get_sdf_storage(self.h, asset, C.byref(b), C.byref(ns), C.byref(nb)))
        return int(b.value), int(ns.value), int(nb.value)

    def get_mass(self, asset: int):
        m, com, I = np.zeros(1), np.zeros(3), np.zeros(9)
        self._check(self.lib.fw_get_mass(self.h, asset, m.ctypes.data, com.ctypes.data, I.ctypes.data))
        return float(m[0]), com, I.reshape(3, 3)

    # -- environments
    def add_env_bodies(self, bodies: np.ndarray, pairs) -> int:
        b = np.ascontiguousarray(bodies, dtype=scenes.BODY_DTYPE)
        p = np.ascontiguousarray(pairs, np.int32).reshape(-1)
        out = C.c_int()
        self._check(self.lib.fw_add_env_bodies(self.h, b.shape[0], b.ctypes.data, b.shape[1],
                                               p.ctypes.data if len(p) else None, len(p) // 2, C.byref(out)))
        return out.value

    def add_pile(self, bodies: np.ndarray, max_pairs: int = 0, max_contacts: int = 0) -> int:
        """One pile env of up to 1024 bodies whose pairs every detection finds again."""
        b = np.ascontiguousarray(bodies, dtype=scenes.BODY_DTYPE).reshape(-1)
        out = C.c_int()
        self._check(self.lib.fw_add_pile(self.h, b.ctypes.data, len(b), max_pairs, max_contacts, C.byref(out)))
        return out.value

    def pile_pairs(self, env: int) -> Tuple[np.ndarray, np.ndarray]:
        """A pile env's current pairs (n x 2 local body ids: sample body, SDF body) and each
        pair's colour in the last solve (-1: no contacts)."""
        cap = 1024
        while True:
            ab, col = np.zeros((cap, 2), np.int32), np.zeros(cap, np.int32)
            n = C.c_int()
            st = self.lib.fw_get_pile_pairs(self.h, env, ab.ctypes.data, col.ctypes.data, cap, C.byref(n))
            if st == -6 and n.value > cap:
                cap = n.value
                continue
            self._check(st)
            return ab[: n.value].copy(), col[: n.value].copy()

    def counts(self) -> Tuple[int, int, int]:
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        self._check(self.lib.fw_get_counts(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def env_info(self, env: int) -> Tuple[int, int, int, int]:
        """(first body, bodies, first pair, pairs) of an env in the world's global order."""
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        self._check(self.lib.fw_get_env_info(self.h, env, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        return a.value, b.value, c.value, d.value

    # -- stepping
    def step(self, n_substeps: int, n_iters: int):
        self._check(self.lib.fw_step(self.h, n_substeps, n_iters))

    def substep(self, hs: float, n_iters: int, detect: bool = True):
        self._check(self.lib.fw_substep(self.h, hs, n_iters, int(detect)))

    def collide(self):
        self._check(self.lib.fw_collide(self.h))

    def sync(self):
        self._check(self.lib.fw_sync(self.h))

    def get_contacts(self, env: int) -> np.ndarray:
        cap = 2048
        while True:
            out = np.zeros(cap, CONTACT_DTYPE)
            n = C.c_int()
            st = self.lib.fw_get_contacts(self.h, env, out.ctypes.data, cap, C.byref(n))
            if st == -6 and n.value > cap:
                cap = n.value
                continue
            self._check(st)
            return out[: n.value].copy()

    def set_contacts(self, env: int, contacts: np.ndarray):
        c = np.ascontiguousarray(contacts, CONTACT_DTYPE)
        self._check(self.lib.fw_set_contacts(self.h, env, c.ctypes.data, len(c)))

    # -- state
    def get_state(self, out=None):
        """(pos, quat, linvel, angvel) as float32 numpy arrays, or fills the given torch
        CUDA tensors (device copies, no synchronisation)."""
        nb = self.counts()[1]
        if out is None:
            p, q = np.zeros((nb, 3), np.float32), np.zeros((nb, 4), np.float32)
            v, w = np.zeros((nb, 3), np.float32), np.zeros((nb, 3), np.float32)
            self._check(self.lib.fw_get_state(self.h, p.ctypes.data, q.ctypes.data, v.ctypes.data,
                                              w.ctypes.data, 0))
            return p, q, v, w
        ptrs = [_ptr(t) for t in out]
        dev = any(d for _, d in ptrs)
        self._check(self.lib.fw_get_state(self.h, *[pp for pp, _ in ptrs], int(dev)))
        return out

    def set_state(self, pos=None, quat=None, linvel=None, angvel=None):
        conv = []
        for a in (pos, quat, linvel, angvel):
            conv.append(a if (a is None or hasattr(a, "data_ptr")) else np.ascontiguousarray(a, np.float32))
        ptrs = [_ptr(a) for a in conv]
        dev = any(d for _, d in ptrs)
        self._check(self.lib.fw_set_state(self.h, *[pp for pp, _ in ptrs], int(dev)))

    # -- test hooks
    def query_sdf(self, asset: int, pts):
        if hasattr(pts, "data_ptr"):
            import torch
            n = pts.shape[0]
            phi = torch.empty(n, device=pts.device, dtype=torch.float32)
            grad = torch.empty((n, 3), device=pts.device, dtype=torch.float32)
            self._check(self.lib.fw_query_sdf(self.h, asset, pts.data_ptr(), n, phi.data_ptr(), grad.data_ptr(), 1))
            return phi, grad
        P = np.ascontiguousarray(pts, np.float32).reshape(-1, 3)
        phi, grad = np.zeros(len(P), np.float32), np.zeros((len(P), 3), np.float32)
        self._check(self.lib.fw_query_sdf(self.h, asset, P.ctypes.data, len(P), phi.ctypes.data,
                                          grad.ctypes.data, 0))
        return phi, grad

    def query_pair(self, env: int, pair: int, n_samples: int):
        phi, nrm = np.zeros(n_samples, np.float32), np.zeros((n_samples, 3), np.float32)
        self._check(self.lib.fw_query_pair(self.h, env, pair, phi.ctypes.data, nrm.ctypes.data, 0))
        return phi, nrm

    def tri_contacts(self, env: int, pair: int, n_tris: int):
        """Per triangle of the pair's point body: minimiser on the face (world), phi (+inf:
        no candidate point), world normal (fw_tri_contacts)."""
        x, nrm = np.zeros((n_tris, 3), np.float32), np.zeros((n_tris, 3), np.float32)
        phi = np.zeros(n_tris, np.float32)
        self._check(self.lib.fw_tri_contacts(self.h, env, pair, x.ctypes.data, phi.ctypes.data, nrm.ctypes.data, 0))
        return x, phi, nrm

    def reduce(self, cands: np.ndarray):
        c = np.ascontiguousarray(cands).view(CANDIDATE_DTYPE)
        cap = 7 * 256
        out = np.zeros(cap, CONTACT_DTYPE)
        n, npch = C.c_int(), C.c_int()
        self._check(self.lib.fw_reduce(self.h, c.ctypes.data if len(c) else None, len(c), out.ctypes.data,
                                       cap, C.byref(n), C.byref(npch)))
        return out[: n.value].copy(), npch.value

    def reduce_noalloc(self, d_cands, n: int, d_out, cap: int, d_counts):
        """fw_reduce_noalloc on device buffers (torch CUDA tensors or raw pointers)."""
        ptr = lambda t: t if isinstance(t, int) else t.data_ptr()
        self._check(self.lib.fw_reduce_noalloc(self.h, ptr(d_cands), n, ptr(d_out), cap, ptr(d_counts)))

    # -- diagnostics
    def set_timing(self, enable: bool):
        self._check(self.lib.fw_set_timing(self.h, int(enable)))

    def get_timings(self):
        ms = np.zeros(6, np.float32)
        self._check(self.lib.fw_get_timings(self.h, ms.ctypes.data, 6))
        return {"detect_ms": float(ms[0]), "solve_ms": float(ms[1]), "detect_launches": int(ms[2]),
                "query_ms": float(ms[4]), "reduce_ms": float(ms[5]),
                "solve_launches": int(ms[3])}

    def set_solve_shape(self, envs_per_warp: int = 0, warps_per_block: int = 0):
        self._check(self.lib.fw_set_solve_shape(self.h, envs_per_warp, warps_per_block))

    def autotune_solve(self, n_substeps: int, n_iters: int, trials: int = 3):
        """times every solve shape on the current state and keeps the fastest:
        (envs_per_warp, warps_per_block, ms per solve launch)"""
        g, w, ms = C.c_int(), C.c_int(), C.c_float()
        self._check(self.lib.fw_autotune_solve(self.h, n_substeps, n_iters, trials, C.byref(g), C.byref(w),
                                               C.byref(ms)))
        return g.value, w.value, ms.value

    def test_stall(self, what: int):
        """test hook: 1 pile grid barriers, 2 solve chunk waits run out (bounded)"""
        self._check(self.lib.fw_test_stall(self.h, what))

    def set_detect_shape(self, query_threads: int = 0, reduce_warps: int = 0):
        self._check(self.lib.fw_set_detect_shape(self.h, query_threads, reduce_warps))

    def set_query_cull(self, on: bool):
        """The narrow phase's bounding-sphere cull of sample groups (on by default; the
        results are the same either way)."""
        self._check(self.lib.fw_set_query_cull(self.h, 1 if on else 0))

    def query_cull(self) -> bool:
        v = C.c_int()
        self._check(self.lib.fw_get_query_cull(self.h, C.byref(v)))
        return bool(v.value)

    def detect_shape(self):
        a, b = C.c_int(), C.c_int()
        self._check(self.lib.fw_get_detect_shape(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def autotune_detect(self, trials: int = 3):
        """(query threads, reduction warps, ms of one query + one reduction launch)"""
        a, b, ms = C.c_int(), C.c_int(), C.c_float()
        self._check(self.lib.fw_autotune_detect(self.h, trials, C.byref(a), C.byref(b), C.byref(ms)))
        return a.value, b.value, ms.value

    def solve_shape(self):
        g, w = C.c_int(), C.c_int()
        self._check(self.lib.fw_get_solve_shape(self.h, C.byref(g), C.byref(w)))
        return g.value, w.value

    def detect_stats(self):
        """(candidates, reduced contacts) of the last detection pass, summed over pairs."""
        a, b = C.c_longlong(), C.c_longlong()
        self._check(self.lib.fw_get_detect_stats(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def launches_per_step(self, n_substeps: int) -> int:
        return self.lib.fw_launches_per_step(self.h, n_substeps)

    # -- differentiable rollout
    def record_rollout(self, n_substeps: int, n_iters: int):
        self._check(self.lib.fw_record_rollout(self.h, n_substeps, n_iters))

    def step_fwd_ckpt(self, n_substeps: int, n_iters: int):
        """One frame forward with its tape and checkpoints (fw_step_fwd_ckpt)."""
        self._check(self.lib.fw_step_fwd_ckpt(self.h, n_substeps, n_iters))

    def replay_rollout(self):
        self._check(self.lib.fw_replay_rollout(self.h))

    def step_bwd(self, g_pos, g_quat, g_linvel, g_angvel):
        """The adjoint of the frame last stepped by step_fwd_ckpt (fw_step_bwd)."""
        return self.adjoint_rollout(g_pos, g_quat, g_linvel, g_angvel, _entry="fw_step_bwd")

    def adjoint_rollout(self, g_pos, g_quat, g_linvel, g_angvel, _entry="fw_adjoint_rollout"):
        """Adjoints of the initial state and parameters of the last record/replay, given
        those of its final state.  numpy in -> numpy out, CUDA tensors in -> CUDA tensors
        out: (pos, quat, linvel, angvel, mass, mu)."""
        nb, npair = self.counts()[1], self.counts()[2]
        dev = hasattr(g_pos, "data_ptr") and g_pos.is_cuda
        if dev:
            import torch
            mk = lambda *shape: torch.zeros(shape, dtype=torch.float32, device=g_pos.device)
            gs = [t.detach().contiguous().float() for t in (g_pos, g_quat, g_linvel, g_angvel)]
        else:
            mk = lambda *shape: np.zeros(shape, np.float32)
            gs = [np.ascontiguousarray(a, np.float32) for a in (g_pos, g_quat, g_linvel, g_angvel)]
        outs = [mk(nb, 3), mk(nb, 4), mk(nb, 3), mk(nb, 3), mk(nb), mk(max(npair, 1))]
        self._check(getattr(self.lib, _entry)(self.h, *[_ptr(a)[0] for a in gs], *[_ptr(a)[0] for a in outs],
                                              int(dev)))
        outs[5] = outs[5][:npair]
        return tuple(outs)

    def get_tape(self):
        info = np.zeros(4, np.int32)
        self._check(self.lib.fw_get_tape(self.h, info.ctypes.data, None, None, None, None))
        S, E, K, n = (int(v) for v in info)
        t = dict(S=S, K=K, c_off=np.zeros(S * E + 1, np.int32), c_rec=np.zeros((max(n, 1), 6), np.int32),
                 r_bits=np.zeros(max(K * n, 1), np.uint8), b_bits=np.zeros(max(S * E, 1), np.uint8))
        self._check(self.lib.fw_get_tape(self.h, info.ctypes.data, t["c_off"].ctypes.data, t["c_rec"].ctypes.data,
                                         t["r_bits"].ctypes.data, t["b_bits"].ctypes.data))
        t["c_rec"], t["r_bits"], t["b_bits"] = t["c_rec"][:n], t["r_bits"][: K * n], t["b_bits"][: S * E]
        return t

    def set_body_params(self, mass=None, mu=None):
        m = None if mass is None else np.ascontiguousarray(mass, np.float32)
        u = None if mu is None else np.ascontiguousarray(mu, np.float32)
        self._check(self.lib.fw_set_body_params(self.h, None if m is None else m.ctypes.data,
                                                None if u is None else u.ctypes.data))


def world_from_scene(scene, fp16: bool = False, stream=None, **over) -> World:
    """Builds a World from a scenes.Scene: assets, SDF bakes, env groups."""
    sim = scene.sim
    cfg = default_config(gravity=sim.gravity, dt=sim.dt, contact_offset=sim.contact_offset,
                         cos_patch=sim.cos_patch, max_patches=sim.max_patches,
                         baumgarte=sim.baumgarte, n_vel_iters=sim.n_vel_iters,
                         max_angvel=sim.max_angvel, sdf_fp16=int(fp16))
    for k, v in over.items():
        if k == "gravity":
            cfg.gravity[:] = list(v)
        else:
            setattr(cfg, k, v)
    if stream is not None:
        cfg.cuda_stream = stream
    w = World(cfg)
    for a in scene.assets:
        i = w.add_mesh_asset(a.verts, a.tris, a.samples, a.density)
        if a.sdf_res:
            w.bake_sdf(i, a.sdf_res, a.sdf_pad, True)
    for g in scene.groups:
        w.add_env_bodies(g.bodies, g.pairs)
    for pb in scene.piles:
        w.add_pile(pb)
    return w


def rollout_function():
    """torch.autograd.Function over a recorded rollout: forward(world, n_substeps, n_iters,
    pos0, quat0, linvel0, angvel0, mass, mu) sets the initial state (n_bodies x 3/4/3/3
    CUDA tensors) and the parameters (mass per body, mu per pair), records the rollout and
    returns the final (pos, quat, linvel, angvel); backward runs fw_adjoint_rollout with the
    incoming gradients and returns those of the initial state, the masses and the mus."""
    import torch

    class Rollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, world, n_substeps, n_iters, pos0, quat0, linvel0, angvel0, mass, mu):
            torch.cuda.synchronize(pos0.device)     # the world copies on its own stream
            world.set_body_params(mass.detach().cpu().numpy(), mu.detach().cpu().numpy())
            world.set_state(*[t.detach().contiguous().float() for t in (pos0, quat0, linvel0, angvel0)])
            world.record_rollout(n_substeps, n_iters)
            nb = world.counts()[1]
            out = [torch.empty((nb, k), dtype=torch.float32, device=pos0.device) for k in (3, 4, 3, 3)]
            world.get_state(out=out)
            torch.cuda.synchronize(pos0.device)
            ctx.world = world
            return tuple(out)

        @staticmethod
        def backward(ctx, gp, gq, gv, gw):
            dev = gp.device if gp is not None else gq.device
            z = lambda t, k: t if t is not None else torch.zeros((ctx.world.counts()[1], k), device=dev)
            torch.cuda.synchronize(dev)
            dp, dq, dv, dw, dm, dmu = ctx.world.adjoint_rollout(z(gp, 3), z(gq, 4), z(gv, 3), z(gw, 3))
            return None, None, None, dp, dq, dv, dw, dm, dmu

    return Rollout

