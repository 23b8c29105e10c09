"""Python binding of libicr (ctypes): argument marshalling only.

Every function here forwards to the C ABI of the same name declared in
include/icr.h; all arithmetic of the constraint-resolution path runs in the
library's CUDA kernels.  The library must have been built
(``paper_2306_06946_gb300.build.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libicr.so")

OK, EINVAL, ENOTSPD, ESTATE, ENOMEM, ENOCONV, ETIMEOUT, ECUDA = range(8)
FP32, FP64 = 0, 1
FIELD = {"WH": 0, "W": 1, "LAMBDA": 2, "P": 3, "DELTA": 4, "C": 5, "MU": 6, "U": 7,
         "REACH_PTR": 8, "REACH_IDX": 9, "DQ": 10, "LAMBDA0": 11}
_INT_FIELDS = {"REACH_PTR", "REACH_IDX"}

# every symbol include/icr.h declares
EXPORTS = ("icr_last_error", "icr_ctx_create", "icr_ctx_destroy", "icr_ctx_bytes_in_use", "icr_scene_create",
           "icr_scene_destroy", "icr_set_params", "icr_set_system", "icr_set_mapping", "icr_set_proximity",
           "icr_reset_proximity", "icr_scene_launches", "icr_update_directions", "icr_set_obstacle_plane", "icr_set_obstacle_sphere",
           "icr_set_obstacle_spheres", "icr_set_step_inputs", "icr_linearize",
           "icr_build_WH", "icr_update_W", "icr_solve_friction", "icr_update_proximity", "icr_correct_motion",
           "icr_get", "icr_field_bytes", "icr_set_field", "icr_reach_noalloc", "icr_step", "icr_step_capture",
           "icr_step_launch", "icr_sync", "icr_serve", "icr_autotune",
           "icr_set_forward_plan", "icr_forward_levels", "icr_build_info",
           "icr_profile_begin", "icr_profile_end",
           "icr_ctx_set_wait_limit", "icr_ctx_inject_alloc_failure", "icr_scene_evict", "icr_scene_readmit",
           "icr_scene_residency", "icr_serve_ex", "icr_newton_iterations", "icr_batch_create", "icr_batch_launch",
           "icr_batch_info", "icr_batch_destroy", "icr_batch_merge_plan", "icr_batch_profile")


class IcrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libicr error {code}: {msg}")
        self.code = code


CONTRACT = {"auto": 0, "simt": 1, "tf32x3": 2, "tf32": 3, "bf16": 4}


W_UPDATE = {"fp32": 0, "tf32": 1, "bf16": 2}


class Params(ct.Structure):
    _fields_ = [("precision", ct.c_int32), ("n_sweeps", ct.c_int32), ("tol", ct.c_double),
                ("contraction", ct.c_int32), ("warm_start", ct.c_int32), ("w_update", ct.c_int32),
                ("newton_tol", ct.c_double)]


class BuildInfo(ct.Structure):
    _fields_ = [("levels", ct.c_int32), ("tc_levels", ct.c_int32), ("gemm_tc_units", ct.c_int32),
                ("gemm_tc_split_max", ct.c_int32), ("gemm_simt_units", ct.c_int32),
                ("contract_tc_units", ct.c_int32), ("contract_tc_split", ct.c_int32),
                ("contract_simt_units", ct.c_int32), ("prox_split", ct.c_int32), ("reach_nnz", ct.c_int64),
                ("flops_front_tc", ct.c_double), ("flops_front_simt", ct.c_double),
                ("flops_contract_tc", ct.c_double), ("flops_contract_simt", ct.c_double),
                ("short_tile_levels", ct.c_int32)]


class ServeStats(ct.Structure):
    _fields_ = [("evictions", ct.c_int32), ("readmissions", ct.c_int32), ("rejected", ct.c_int32),
                ("admit_s", ct.c_double)]


class BatchInfo(ct.Structure):
    _fields_ = [("n_scenes", ct.c_int32), ("n_groups", ct.c_int32), ("launches_per_step", ct.c_int32),
                ("kernel_launches_per_step", ct.c_int32), ("scene_launches_per_step", ct.c_int64),
                ("argument_bytes", ct.c_uint64), ("steps", ct.c_uint64)]


class BatchLaunchTime(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("group", ct.c_int32), ("slots", ct.c_int32), ("blocks", ct.c_int32),
                ("ms", ct.c_double)]


class KernelTime(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("launches", ct.c_int32), ("total_ms", ct.c_double)]


class PgsStats(ct.Structure):
    _fields_ = [("sweeps", ct.c_int32), ("n_separated", ct.c_int32), ("n_stick", ct.c_int32),
                ("n_slip", ct.c_int32), ("eps", ct.c_double), ("res_normal", ct.c_double),
                ("res_cone", ct.c_double), ("res_stick", ct.c_double), ("res_slip", ct.c_double),
                ("sweeps_s_only", ct.c_int32), ("deferred_folds", ct.c_int32), ("rechecks", ct.c_int32),
                ("joins", ct.c_int32)]


_lib = None
P = ct.c_void_p


def lib() -> ct.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2306_06946_gb300.build.build()")
        L = ct.CDLL(LIB_PATH)
        L.icr_last_error.restype = ct.c_char_p
        L.icr_last_error.argtypes = []
        sigs = {
            "icr_ctx_create": [ct.POINTER(P), ct.c_int, P, ct.c_uint64],
            "icr_ctx_destroy": [P],
            "icr_ctx_bytes_in_use": [P, ct.POINTER(ct.c_uint64)],
            "icr_ctx_set_wait_limit": [P, ct.c_uint64],
            "icr_ctx_inject_alloc_failure": [P, ct.c_int64],
            "icr_scene_create": [P, ct.POINTER(P), ct.POINTER(Params)],
            "icr_scene_destroy": [P],
            "icr_set_params": [P, ct.POINTER(Params)],
            "icr_set_system": [P, ct.c_int32, ct.c_int32, P, P, P, P, P, P, P],
            "icr_set_mapping": [P, ct.c_int32, P, P],
            "icr_set_proximity": [P, P],
            "icr_reset_proximity": [P],
            "icr_scene_launches": [P, ct.POINTER(ct.c_uint64)],
            "icr_update_directions": [P, P, P, P],
            "icr_set_obstacle_plane": [P, ct.c_int32, P, P],
            "icr_set_obstacle_sphere": [P, P, ct.c_double, P],
            "icr_set_obstacle_spheres": [P, ct.c_int32, P, P, P],
            "icr_set_step_inputs": [P, ct.c_int32, P, P, P, P, ct.c_int32, P, P, P],
            "icr_linearize": [P, ct.c_int32],
            "icr_build_WH": [P],
            "icr_update_W": [P],
            "icr_solve_friction": [P, ct.c_int, ct.POINTER(PgsStats)],
            "icr_update_proximity": [P, P],
            "icr_correct_motion": [P, P, ct.c_int],
            "icr_get": [P, ct.c_int32, P, ct.c_size_t],
            "icr_field_bytes": [P, ct.c_int32, ct.POINTER(ct.c_size_t)],
            "icr_set_field": [P, ct.c_int32, P, ct.c_size_t],
            "icr_reach_noalloc": [ct.c_int32, ct.c_int32, ct.c_int32, P, P, P, P, P, P],
            "icr_step": [P, ct.c_int32],
            "icr_newton_iterations": [P, ct.POINTER(ct.c_int32)],
            "icr_step_capture": [P, ct.c_int32],
            "icr_step_launch": [P],
            "icr_sync": [P],
            "icr_autotune": [P, P, P, ct.c_int32],
            "icr_set_forward_plan": [P, P, ct.c_int32],
            "icr_forward_levels": [P, P],
            "icr_build_info": [P, ct.POINTER(BuildInfo)],
            "icr_profile_begin": [P],
            "icr_profile_end": [P, ct.POINTER(KernelTime), ct.c_int32, ct.POINTER(ct.c_int32)],
            "icr_serve": [ct.POINTER(P), ct.c_int32, P, P, ct.c_int32, ct.c_int32, ct.c_double, P, P],
            "icr_serve_ex": [ct.POINTER(P), ct.c_int32, P, P, ct.c_int32, ct.c_int32, ct.c_double, P, P,
                             ct.POINTER(ServeStats)],
            "icr_scene_evict": [P],
            "icr_scene_readmit": [P],
            "icr_scene_residency": [P, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_uint64)],
            "icr_batch_create": [ct.POINTER(P), ct.POINTER(P), ct.c_int32, ct.c_int32, ct.c_int32],
            "icr_batch_launch": [P],
            "icr_batch_info": [P, ct.POINTER(BatchInfo)],
            "icr_batch_destroy": [P],
            "icr_batch_profile": [P, ct.POINTER(BatchLaunchTime), ct.c_int32, ct.POINTER(ct.c_int32)],
            "icr_batch_merge_plan": [P, P, ct.c_int32, P, P, P, ct.c_int32, P],
        }
        for name, args in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ct.c_int
        _lib = L
    return _lib


def _check(code: int):
    if code != OK:
        raise IcrError(code, lib().icr_last_error().decode())


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(P)


def _arr(x, dtype, shape=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
    if shape is not None:
        a = a.reshape(shape)
    return a


NOALLOC_SCRATCH_WORDS = 1 << 20


def reach_noalloc(m: int, nsuper: int, n_nodes: int, nodes_ptr: int, node_super_ptr: int, parent_ptr: int,
                  qcount_ptr: int, qidx_ptr: int, stream: int = 0) -> None:
    """icr_reach_noalloc: every argument after the sizes is a raw device
    address owned by the caller; the library allocates nothing."""
    _check(lib().icr_reach_noalloc(int(m), int(nsuper), int(n_nodes), P(nodes_ptr or None),
                                   P(node_super_ptr or None), P(parent_ptr or None), P(qcount_ptr or None),
                                   P(qidx_ptr or None), P(stream or None)))


def serve(scenes, req_scene, req_arrival_s, n_slots: int, timeout_s: float = 120.0, stats: bool = False):
    """icr_serve_ex: returns (latency_s per request, makespan_s), and with
    ``stats`` also a dict of evictions, readmissions, rejections and admit_s."""
    arr = (P * len(scenes))(*[sc.h for sc in scenes])
    rs = _arr(req_scene, np.int32)
    ra = _arr(req_arrival_s, np.float64)
    lat = np.zeros(rs.size)
    mk = ct.c_double()
    st = ServeStats()
    _check(lib().icr_serve_ex(arr, len(scenes), _ptr(rs), _ptr(ra), int(rs.size), int(n_slots), float(timeout_s),
                              _ptr(lat), ct.byref(mk), ct.byref(st)))
    if stats:
        return lat, float(mk.value), {f: getattr(st, f) for f, _ in ServeStats._fields_}
    return lat, float(mk.value)


class Context:
    """icr_ctx: one device, one CUDA stream (a raw cudaStream_t handle, 0 for
    the legacy default stream) and an HBM budget in bytes (0 = none)."""

    def __init__(self, device: int = 0, stream: int = 0, hbm_budget: int = 0):
        h = P()
        _check(lib().icr_ctx_create(ct.byref(h), device, P(stream or None), hbm_budget))
        self.h = h

    @classmethod
    def on_torch_stream(cls, device: int = 0, hbm_budget: int = 0):
        import torch
        return cls(device, torch.cuda.current_stream(device).cuda_stream, hbm_budget)

    def bytes_in_use(self) -> int:
        v = ct.c_uint64()
        _check(lib().icr_ctx_bytes_in_use(self.h, ct.byref(v)))
        return int(v.value)

    def set_wait_limit(self, ns: int):
        """Bound of the tensor-core pipeline waits in ns (0: one poll, failure injection)."""
        _check(lib().icr_ctx_set_wait_limit(self.h, int(ns)))

    def inject_alloc_failure(self, after: int):
        """The allocation after the next ``after`` ones fails once (-1: off)."""
        _check(lib().icr_ctx_inject_alloc_failure(self.h, int(after)))

    def close(self):
        if self.h:
            lib().icr_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_merge_plan(sequences):
    """icr_batch_merge_plan (host only): the merged launches of integer key
    sequences, as a list of (key, [indices of the sequences it covers])."""
    lens = _arr([len(q) for q in sequences], np.int32)
    keys = _arr([k for q in sequences for k in q] or [0], np.int32)
    total = int(lens.sum())
    out_key = np.zeros(max(total, 1), np.int32)
    out_count = np.zeros(max(total, 1), np.int32)
    out_cover = np.zeros(max(total, 1), np.int32)
    n = ct.c_int32()
    _check(lib().icr_batch_merge_plan(_ptr(keys), _ptr(lens), len(sequences), _ptr(out_key),
                                      _ptr(out_count), _ptr(out_cover), int(out_key.size), ct.byref(n)))
    res, c = [], 0
    for i in range(n.value):
        res.append((int(out_key[i]), out_cover[c:c + out_count[i]].tolist()))
        c += int(out_count[i])
    return res


class Batch:
    """icr_batch: many scenes of one context stepped together by one captured
    graph whose every kernel launch covers all of them.  Creating it runs one
    batched step; every launch() runs one more time step of every scene."""

    def __init__(self, scenes, n_newton: int, n_groups: int = 1):
        self.scenes = list(scenes)   # kept alive while the batch holds them
        arr = (P * len(self.scenes))(*[sc.h for sc in self.scenes])
        h = P()
        _check(lib().icr_batch_create(ct.byref(h), arr, len(self.scenes), int(n_newton), int(n_groups)))
        self.h = h

    def launch(self):
        _check(lib().icr_batch_launch(self.h))

    def info(self) -> dict:
        bi = BatchInfo()
        _check(lib().icr_batch_info(self.h, ct.byref(bi)))
        return {f: getattr(bi, f) for f, _ in BatchInfo._fields_}

    def profile(self) -> list[dict]:
        """One eager batched step with CUDA events around every merged launch."""
        n = ct.c_int32()
        size = max(1, self.info()["launches_per_step"])
        arr = (BatchLaunchTime * size)()
        _check(lib().icr_batch_profile(self.h, arr, size, ct.byref(n)))
        return [{"name": a.name.decode(), "group": a.group, "slots": a.slots, "blocks": a.blocks, "ms": a.ms}
                for a in arr[:n.value]]

    def close(self):
        if getattr(self, "h", None):
            lib().icr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scene:
    """icr_scene: one deformable body and its contacts."""

    def __init__(self, ctx: Context, precision: int = FP32, n_sweeps: int = 50, tol: float = 0.0,
                 contraction: str = "auto", warm_start: bool = False, w_update: str = "fp32",
                 newton_tol: float = 0.0):
        self.ctx = ctx
        self.params = Params(precision, n_sweeps, tol, CONTRACT[contraction], int(bool(warm_start)),
                             W_UPDATE[w_update], float(newton_tol))
        h = P()
        _check(lib().icr_scene_create(ctx.h, ct.byref(h), ct.byref(self.params)))
        self.h = h
        self.n = 0
        self.m = 0

    def close(self):
        if getattr(self, "h", None):
            _check(lib().icr_scene_destroy(self.h))   # refused (ICR_ESTATE) while a batch holds the scene
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, n_sweeps: int | None = None, tol: float | None = None, contraction: str | None = None,
                   warm_start: bool | None = None, w_update: str | None = None, newton_tol: float | None = None):
        if w_update is not None:
            self.params.w_update = W_UPDATE[w_update]
        if newton_tol is not None:
            self.params.newton_tol = float(newton_tol)
        if warm_start is not None:
            self.params.warm_start = int(bool(warm_start))
        if n_sweeps is not None:
            self.params.n_sweeps = n_sweeps
        if tol is not None:
            self.params.tol = tol
        if contraction is not None:
            self.params.contraction = CONTRACT[contraction]
        _check(lib().icr_set_params(self.h, ct.byref(self.params)))

    def set_system(self, n, super_ptr, rowpat_ptr, rowpat, val_ptr, Lpanels, D, parent):
        sp = _arr(super_ptr, np.int32)
        rp = _arr(rowpat_ptr, np.int64)
        rw = _arr(rowpat, np.int32)
        vp = _arr(val_ptr, np.int64)
        Lv = _arr(Lpanels, np.float64)
        Dv = _arr(D, np.float64)
        pa = _arr(parent, np.int32)
        _check(lib().icr_set_system(self.h, int(n), int(sp.size - 1), _ptr(sp), _ptr(rp), _ptr(rw), _ptr(vp),
                                    _ptr(Lv), _ptr(Dv), _ptr(pa)))
        self.n = int(n)

    def set_mapping(self, nodes, bary):
        nd = _arr(nodes, np.int32).reshape(-1, 4)
        bw = _arr(bary, np.float64).reshape(-1, 4)
        _check(lib().icr_set_mapping(self.h, int(nd.shape[0]), _ptr(nd), _ptr(bw)))
        self.m = int(nd.shape[0])

    def set_proximity(self, p):
        _check(lib().icr_set_proximity(self.h, _ptr(_arr(p, np.float64))))

    def reset_proximity(self):
        _check(lib().icr_reset_proximity(self.h))

    def launches(self) -> int:
        v = ct.c_uint64()
        _check(lib().icr_scene_launches(self.h, ct.byref(v)))
        return int(v.value)

    def update_directions(self, C, delta, mu=None):
        mu_a = None if mu is None else _arr(mu, np.float64)
        _check(lib().icr_update_directions(self.h, _ptr(_arr(C, np.float64)), _ptr(_arr(delta, np.float64)),
                                           _ptr(mu_a)))

    def set_obstacle_plane(self, normals, anchors):
        nr = _arr(normals, np.float64)
        _check(lib().icr_set_obstacle_plane(self.h, int(nr.size // max(1, 3 * self.m)) if self.m else 1,
                                            _ptr(nr), _ptr(_arr(anchors, np.float64))))

    def set_obstacle_sphere(self, center, radius, anchors):
        _check(lib().icr_set_obstacle_sphere(self.h, _ptr(_arr(center, np.float64)), float(radius),
                                             _ptr(_arr(anchors, np.float64))))

    def set_obstacle_spheres(self, spheres, contact_sphere, anchors):
        sp = _arr(spheres, np.float64).reshape(-1, 4)
        _check(lib().icr_set_obstacle_spheres(self.h, int(sp.shape[0]), _ptr(sp),
                                              _ptr(_arr(contact_sphere, np.int32)), _ptr(_arr(anchors, np.float64))))

    def set_step_inputs(self, nodes, bary, p0, mu, spheres, contact_sphere, anchors):
        """A time step's inputs in one call (mapping, proximity positions, sphere
        tools, friction): one host-to-device copy when the contact count is
        unchanged."""
        nd = _arr(nodes, np.int32).reshape(-1, 4)
        sp = _arr(spheres, np.float64).reshape(-1, 4)
        _check(lib().icr_set_step_inputs(self.h, int(nd.shape[0]), _ptr(nd), _ptr(_arr(bary, np.float64)),
                                         _ptr(_arr(p0, np.float64)), _ptr(_arr(mu, np.float64)), int(sp.shape[0]),
                                         _ptr(sp), _ptr(_arr(contact_sphere, np.int32)),
                                         _ptr(_arr(anchors, np.float64))))
        self.m = int(nd.shape[0])

    def linearize(self, k: int):
        _check(lib().icr_linearize(self.h, int(k)))

    def build_WH(self):
        _check(lib().icr_build_WH(self.h))

    def update_W(self):
        _check(lib().icr_update_W(self.h))

    def solve_friction(self, warm_start: bool = False, stats: bool = False):
        """Returns None, or a dict of the FP64 stats when ``stats``; a run that
        stops above a positive tol reports converged=False instead of raising."""
        if not stats:
            _check(lib().icr_solve_friction(self.h, int(bool(warm_start)), None))
            return None
        st = PgsStats()
        code = lib().icr_solve_friction(self.h, int(bool(warm_start)), ct.byref(st))
        if code not in (OK, ENOCONV):
            _check(code)
        out = {f: getattr(st, f) for f, _ in PgsStats._fields_}
        out["converged"] = code == OK
        return out

    def update_proximity(self, want_dp: bool = False):
        if not want_dp:
            _check(lib().icr_update_proximity(self.h, None))
            return None
        dp = np.empty(3 * self.m)
        _check(lib().icr_update_proximity(self.h, _ptr(dp)))
        return dp

    def correct_motion(self, want_dq: bool = True, reset: bool = True, out: np.ndarray | None = None):
        dq = None
        if want_dq:
            dq = out if out is not None else np.empty(self.n)
        _check(lib().icr_correct_motion(self.h, _ptr(dq), int(bool(reset))))
        return dq

    def step(self, n_newton: int):
        _check(lib().icr_step(self.h, int(n_newton)))

    def newton_iterations(self) -> int:
        v = ct.c_int32()
        _check(lib().icr_newton_iterations(self.h, ct.byref(v)))
        return int(v.value)

    def autotune(self, level_times: bool = False):
        """Per-level choice of the forward-solve tile shape; returns the number
        of levels on the tensor cores (and, with ``level_times``, an array of
        [64-row CUDA-core ms, 32-row CUDA-core ms, tensor-core ms] per etree
        level)."""
        n = ct.c_int32(0)
        nlev = self.forward_levels()
        lv = np.zeros(3 * nlev) if level_times else None
        _check(lib().icr_autotune(self.h, ct.byref(n), _ptr(lv), nlev if level_times else 0))
        if not level_times:
            return int(n.value)
        return int(n.value), lv.reshape(nlev, 3)

    def forward_levels(self) -> int:
        n = ct.c_int32(0)
        _check(lib().icr_forward_levels(self.h, ct.byref(n)))
        return int(n.value)

    def set_forward_plan(self, tc_levels):
        f = _arr(tc_levels, np.uint8)
        _check(lib().icr_set_forward_plan(self.h, _ptr(f), int(f.size)))

    def evict(self):
        """icr_scene_evict: keep the scene's state in pinned host memory, free its device memory."""
        _check(lib().icr_scene_evict(self.h))

    def readmit(self):
        _check(lib().icr_scene_readmit(self.h))

    def residency(self):
        """(resident, device bytes held, or held again once readmitted)."""
        r, b = ct.c_int32(), ct.c_uint64()
        _check(lib().icr_scene_residency(self.h, ct.byref(r), ct.byref(b)))
        return bool(r.value), int(b.value)

    def build_info(self) -> dict:
        """Which paths the last W_H build took (icr_build_info)."""
        b = BuildInfo()
        _check(lib().icr_build_info(self.h, ct.byref(b)))
        return {f: (float if f.startswith("flops") else int)(getattr(b, f)) for f, _ in BuildInfo._fields_}

    def profile_begin(self):
        """Time every kernel this scene launches eagerly from now on."""
        _check(lib().icr_profile_begin(self.h))

    def profile_end(self) -> dict:
        """{kernel name: (launches, total device ms)} since profile_begin."""
        buf = (KernelTime * 64)()
        n = ct.c_int32(0)
        _check(lib().icr_profile_end(self.h, buf, 64, ct.byref(n)))
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(64, n.value))}

    def step_capture(self, n_newton: int):
        _check(lib().icr_step_capture(self.h, int(n_newton)))

    def step_launch(self):
        _check(lib().icr_step_launch(self.h))

    def sync(self):
        _check(lib().icr_sync(self.h))

    def field_bytes(self, field: str) -> int:
        v = ct.c_size_t()
        _check(lib().icr_field_bytes(self.h, FIELD[field], ct.byref(v)))
        return int(v.value)

    def get(self, field: str, out: np.ndarray | None = None) -> np.ndarray:
        """Copy a field to the host (into ``out`` when given: a contiguous
        array of the field's dtype and size, e.g. pinned memory)."""
        nb = self.field_bytes(field)
        dt = np.int32 if field in _INT_FIELDS else np.float64
        if out is None:
            a = np.empty(nb // np.dtype(dt).itemsize, dtype=dt)
        else:
            a = out
            if a.dtype != dt or a.nbytes != nb or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"out must be a contiguous {np.dtype(dt).name} array of {nb} bytes")
        _check(lib().icr_get(self.h, FIELD[field], _ptr(a), nb))
        if field in ("WH", "W"):
            a = a.reshape(3 * self.m, 3 * self.m)
        elif field == "C":
            a = a.reshape(self.m, 3, 3)
        elif field == "P":
            a = a.reshape(self.m, 3)
        return a

    def set_field(self, field: str, values):
        v = _arr(values, np.float64)
        _check(lib().icr_set_field(self.h, FIELD[field], _ptr(v), v.nbytes))
