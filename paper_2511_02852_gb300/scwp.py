"""Python binding of the C ABI in ``include/scwp.h`` (ctypes).

Argument marshalling only: every step of the hybrid-ocean path runs in the
CUDA library ``_lib/libscwp.so``.  There is no fallback: if the library is
missing or cannot be loaded, :func:`lib` raises.  PyTorch, when used, only
supplies device memory (an allocator callback over its caching allocator)
and the stream.

The functions below carry the C names (``scwp_create``, ``scwp_step``, ...)
and take/return ctypes objects; :class:`Scene` is a thin convenience wrapper
used by the tests and the bench.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

MAX_BUCKETS = 64
WAKE_DIRS = 4096
FIELD_H, FIELD_DX, FIELD_DY = 0, 1, 2
SYNTH_GATHER, SYNTH_LAYERED, SYNTH_GATHER_FP32, SYNTH_GATHER_FP16, SYNTH_SAT = 0, 1, 2, 3, 4
(TAB_OMEGA, TAB_K, TAB_C, TAB_R, TAB_E, TAB_EDGES, TAB_AMP, TAB_RQ, TAB_VX, TAB_VY, TAB_QX,
 TAB_QY, TAB_WAKE_VX, TAB_WAKE_VY, TAB_WAKE_QX, TAB_WAKE_QY, TAB_CARRY) = range(17)
STATUS = {0: "SCWP_OK", 1: "SCWP_E_INVALID", 2: "SCWP_E_NOMEM", 3: "SCWP_E_CAPACITY",
          4: "SCWP_E_CUDA", 5: "SCWP_E_TIMEOUT", 6: "SCWP_E_STATE"}
# the status of scwp_stats_get that still fills the statistics: the frame's
# error flags say what happened (bit 0: pool full, injection truncated)
_STATS_FLAGGED = (3,)

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class scwp_spectrum_desc(C.Structure):
    _fields_ = [("spectrum", C.c_int32), ("spreading", C.c_int32),
                ("wind_speed", C.c_double), ("fetch", C.c_double), ("depth", C.c_double),
                ("wind_dir", C.c_double), ("gamma", C.c_double),
                ("n_buckets", C.c_int32), ("n_theta", C.c_int32),
                ("bucket_edges", C.POINTER(C.c_double)),
                ("omega_lo_mul", C.c_double), ("omega_hi_mul", C.c_double),
                ("amp_mode", C.c_int32), ("fft_n", C.c_int32), ("fft_L", C.c_double),
                ("choppiness", C.c_double), ("seed", C.c_uint64),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("stream", C.c_void_p)]


class scwp_patch_desc(C.Structure):
    _fields_ = [("origin_x", C.c_double), ("origin_y", C.c_double), ("cell", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32), ("band", C.c_double),
                ("max_particles", C.c_int32), ("prefill", C.c_int32),
                ("inject_scale", C.c_double), ("bin_cells", C.c_int32), ("emitter", C.c_int32),
                ("obj_radius", C.c_double), ("obj_speed", C.c_double),
                ("obj_path_radius", C.c_double), ("wake_amp", C.c_double),
                ("wake_rate", C.c_int32), ("n_buckets", C.c_int32),
                ("heave_period", C.c_double), ("ring_rate", C.c_int32)]


class scwp_stats(C.Structure):
    _fields_ = [("frame", C.c_int64), ("time", C.c_double), ("live_particles", C.c_int64),
                ("bumps_binned", C.c_int64), ("eval_count", C.c_int64),
                ("injected_total", C.c_int64), ("n_buckets", C.c_int32),
                ("error_flags", C.c_int32), ("live_per_bucket", C.c_int64 * MAX_BUCKETS),
                ("injected_energy", C.c_double * MAX_BUCKETS), ("mma_stages", C.c_int64),
                ("eval_total", C.c_int64), ("sat_candidates", C.c_int64)]


class scwp_patch_info(C.Structure):
    _fields_ = [("n_buckets", C.c_int32), ("n_theta", C.c_int32), ("n_dirs", C.c_int32),
                ("wake_bucket", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("total_bins", C.c_int32), ("capacity", C.c_int32),
                ("bin_cells", C.c_int32 * MAX_BUCKETS), ("nbx", C.c_int32 * MAX_BUCKETS),
                ("nby", C.c_int32 * MAX_BUCKETS), ("bin_base", C.c_int32 * MAX_BUCKETS),
                ("synth_groups", C.c_int32), ("synth_items", C.c_int32), ("synth_slots", C.c_int32),
                ("sat_groups", C.c_int32), ("sat_items", C.c_int32), ("sat_slots", C.c_int32),
                ("frame_param_bytes", C.c_int32), ("sat_variant", C.c_int32), ("sat_parts", C.c_int32)]


TUNE_MAX = 8


class scwp_tune_result(C.Structure):
    _fields_ = [("n_configs", C.c_int32), ("chosen", C.c_int32), ("from_cache", C.c_int32),
                ("pad", C.c_int32), ("variant", C.c_int32 * TUNE_MAX), ("gmul", C.c_double * TUNE_MAX),
                ("ms", C.c_double * TUNE_MAX)]


class scwp_server_desc(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("hbm_budget_bytes", C.c_int64), ("max_inflight", C.c_int32),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p)]


class scwp_server_info(C.Structure):
    _fields_ = [("scenes", C.c_int32), ("frames_in_flight", C.c_int32), ("ticks_in_flight", C.c_int32),
                ("pad", C.c_int32), ("pending_requests", C.c_int64), ("device_bytes", C.c_int64),
                ("budget_bytes", C.c_int64), ("ticks_launched", C.c_int64), ("requests_done", C.c_int64)]


EXPORTS = {
    "scwp_create": (C.c_int, [C.POINTER(scwp_spectrum_desc), C.POINTER(C.c_void_p)]),
    "scwp_add_patch": (C.c_int, [C.c_void_p, C.POINTER(scwp_patch_desc), C.POINTER(C.c_int32)]),
    "scwp_step": (C.c_int, [C.c_void_p, C.c_double]),
    "scwp_height_map": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t, C.c_int32]),
    "scwp_height_maps": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t, C.c_int32]),
    "scwp_stats_get": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(scwp_stats)]),
    "scwp_patch_info_get": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(scwp_patch_info)]),
    "scwp_get_table": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t]),
    "scwp_host_table": (C.c_int, [C.POINTER(scwp_spectrum_desc), C.POINTER(scwp_patch_desc),
                                  C.c_double, C.c_int32, C.c_void_p, C.c_size_t,
                                  C.POINTER(C.c_int64)]),
    "scwp_get_particles": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_int64, C.POINTER(C.c_int64)]),
    "scwp_set_particles": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_int64]),
    "scwp_get_bins": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_int64, C.POINTER(C.c_int64)]),
    "scwp_debug_sort_timeout": (C.c_int, [C.c_void_p, C.c_int32, C.c_double]),
    "scwp_resynthesize": (C.c_int, [C.c_void_p, C.c_int32]),
    "scwp_set_synth_mode": (C.c_int, [C.c_void_p, C.c_int32]),
    "scwp_set_batched": (C.c_int, [C.c_void_p, C.c_int32]),
    "scwp_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(scwp_tune_result)]),
    "scwp_set_sat_plan": (C.c_int, [C.c_void_p, C.c_int32, C.c_double]),
    "scwp_set_bucket_range": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "scwp_normal_map": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t, C.c_int32]),
    "scwp_set_timing": (C.c_int, [C.c_void_p, C.c_int32]),
    "scwp_timing_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "scwp_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "scwp_background_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double,
                                          C.c_double, C.c_double, C.c_void_p, C.c_void_p]),
    "scwp_last_error": (C.c_char_p, [C.c_void_p]),
    "scwp_version": (C.c_char_p, []),
    "scwp_destroy": (None, [C.c_void_p]),
    "scwp_server_create": (C.c_int, [C.POINTER(scwp_server_desc), C.POINTER(C.c_void_p)]),
    "scwp_server_add_scene": (C.c_int, [C.c_void_p, C.POINTER(scwp_spectrum_desc), C.c_void_p, C.c_int32,
                                        C.POINTER(C.c_int32)]),
    "scwp_server_remove_scene": (C.c_int, [C.c_void_p, C.c_int32]),
    "scwp_server_submit": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_int64]),
    "scwp_server_tick": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "scwp_server_poll": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "scwp_server_scene": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "scwp_server_info_get": (C.c_int, [C.c_void_p, C.POINTER(scwp_server_info)]),
    "scwp_server_last_error": (C.c_char_p, [C.c_void_p]),
    "scwp_server_destroy": (None, [C.c_void_p]),
}

_lib = None


def lib(path=None, build_if_missing=True):
    """Load libscwp.so (building it in-tree first if it is missing)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        if not build_if_missing:
            raise OSError(f"CUDA library not built: {p}")
        p = _build.build()
    L = C.CDLL(p)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = L
    return L


class ScwpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(status, ctx=None):
    if status != 0:
        msg = lib().scwp_last_error(ctx).decode() if ctx else ""
        raise ScwpError(status, msg)


# -- the C calls, same names ---------------------------------------------------
def scwp_create(desc):
    out = C.c_void_p()
    _check(lib().scwp_create(C.byref(desc), C.byref(out)))
    return out


def scwp_add_patch(ctx, desc):
    pid = C.c_int32()
    _check(lib().scwp_add_patch(ctx, C.byref(desc), C.byref(pid)), ctx)
    return pid.value


def scwp_step(ctx, dt):
    _check(lib().scwp_step(ctx, dt), ctx)


def scwp_height_map(ctx, patch_id, field, dst_ptr, dst_elems, dst_on_device):
    _check(lib().scwp_height_map(ctx, patch_id, field, dst_ptr, dst_elems, dst_on_device), ctx)


def scwp_height_maps(ctx, patch_id, dst_ptr, dst_elems, dst_on_device):
    _check(lib().scwp_height_maps(ctx, patch_id, dst_ptr, dst_elems, dst_on_device), ctx)


def scwp_stats_get(ctx, patch_id):
    st = scwp_stats()
    rc = lib().scwp_stats_get(ctx, patch_id, C.byref(st))
    if rc not in _STATS_FLAGGED:
        _check(rc, ctx)
    return st


def scwp_patch_info_get(ctx, patch_id):
    info = scwp_patch_info()
    _check(lib().scwp_patch_info_get(ctx, patch_id, C.byref(info)), ctx)
    return info


def scwp_destroy(ctx):
    lib().scwp_destroy(ctx)


# -- descriptors from workload dictionaries -------------------------------------
def spectrum_desc(cfg, stream=None, alloc=None, free=None):
    d = scwp_spectrum_desc()
    for k in ("spectrum", "spreading", "n_buckets", "n_theta", "amp_mode", "fft_n"):
        setattr(d, k, int(cfg[k]))
    for k in ("wind_speed", "fetch", "depth", "wind_dir", "gamma", "omega_lo_mul",
              "omega_hi_mul", "fft_L", "choppiness"):
        setattr(d, k, float(cfg[k]))
    d.seed = int(cfg["seed"])
    edges = cfg.get("bucket_edges")
    keep = None
    if edges is not None:
        keep = (C.c_double * len(edges))(*[float(e) for e in edges])
        d.bucket_edges = C.cast(keep, C.POINTER(C.c_double))
    if alloc is not None:
        d.alloc = alloc
        d.free = free
    d.stream = stream
    d._keep = keep
    return d


def patch_desc(p):
    d = scwp_patch_desc()
    for k in ("width", "height", "max_particles", "prefill", "bin_cells", "emitter", "wake_rate",
              "n_buckets", "ring_rate"):
        setattr(d, k, int(p.get(k, 0)))
    for k in ("origin_x", "origin_y", "cell", "band", "inject_scale", "obj_radius", "obj_speed",
              "obj_path_radius", "wake_amp"):
        setattr(d, k, float(p[k]))
    d.heave_period = float(p.get("heave_period", 0.0))
    return d


_TABLE_DTYPES = {TAB_OMEGA: np.float64, TAB_K: np.float64, TAB_C: np.float64, TAB_R: np.float64,
                 TAB_E: np.float64, TAB_EDGES: np.float64, TAB_AMP: np.float64,
                 TAB_RQ: np.int32, TAB_VX: np.int32, TAB_VY: np.int32, TAB_QX: np.int32,
                 TAB_QY: np.int32, TAB_WAKE_VX: np.int32, TAB_WAKE_VY: np.int32,
                 TAB_WAKE_QX: np.int32, TAB_WAKE_QY: np.int32, TAB_CARRY: np.float64}


def scwp_host_table(spec_cfg, patch_cfg, dt, table):
    """Host-only table computation (no GPU): returns a numpy array."""
    sd = spectrum_desc(spec_cfg)
    pd = patch_desc(patch_cfg)
    n = C.c_int64()
    _check(lib().scwp_host_table(C.byref(sd), C.byref(pd), dt, table, None, 0, C.byref(n)))
    out = np.zeros(n.value, dtype=_TABLE_DTYPES[table])
    _check(lib().scwp_host_table(C.byref(sd), C.byref(pd), dt, table,
                                 out.ctypes.data_as(C.c_void_p), out.nbytes, C.byref(n)))
    return out


class Scene:
    """A context with its patches; device memory from torch's caching
    allocator, work on torch's current stream (or a given one)."""

    def __init__(self, scene_cfg, device=0, stream=None, use_torch_alloc=True):
        import torch
        self.torch = torch
        self.cfg = scene_cfg
        self.device = device
        torch.cuda.set_device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._alloc = self._free = None
        if use_torch_alloc:
            st = self.stream

            def _a(nbytes, user):
                try:
                    return int(torch.cuda.caching_allocator_alloc(int(nbytes), device, st))
                except Exception:
                    return None

            def _f(ptr, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._alloc = ALLOC_FN(_a)
            self._free = FREE_FN(_f)
        self.sdesc = spectrum_desc(scene_cfg["spectrum"], C.c_void_p(self.stream.cuda_stream),
                                   self._alloc, self._free)
        self.ctx = scwp_create(self.sdesc)
        self.pids = [scwp_add_patch(self.ctx, patch_desc(p)) for p in scene_cfg["patches"]]
        self.N = int(scene_cfg["spectrum"]["fft_n"])

    def close(self):
        if self.ctx:
            scwp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, dt=None):
        scwp_step(self.ctx, float(dt if dt is not None else self.cfg.get("dt", 1 / 60)))

    def patch_shape(self, p):
        pc = self.cfg["patches"][p]
        return int(pc["height"]), int(pc["width"])

    def maps(self, p):
        """Blended (h, Dx, Dy) of patch p (or the background for p = -1) as
        host float32 arrays."""
        shape = (self.N, self.N) if p == -1 else self.patch_shape(p)
        a = np.empty((3,) + shape, dtype=np.float32)
        scwp_height_maps(self.ctx, p, a.ctypes.data_as(C.c_void_p), a.size, 0)
        return [a[0], a[1], a[2]]

    def maps_device(self, p, out):
        """Copy the maps into a device tensor out[3][H][W] (stream-ordered)."""
        n = out[0].numel()
        for f in range(3):
            scwp_height_map(self.ctx, p, f, C.c_void_p(out[f].data_ptr()), n, 1)

    def stats(self, p=0):
        return scwp_stats_get(self.ctx, p)

    def info(self, p=0):
        return scwp_patch_info_get(self.ctx, p)

    def table(self, p, table):
        info = self.info(p)
        nb, nth = info.n_buckets, info.n_theta
        sizes = {TAB_EDGES: nb + 1, TAB_AMP: nb * nth, TAB_VX: nb * nth, TAB_VY: nb * nth,
                 TAB_QX: nb * nth, TAB_QY: nb * nth, TAB_WAKE_VX: WAKE_DIRS,
                 TAB_WAKE_VY: WAKE_DIRS, TAB_WAKE_QX: WAKE_DIRS, TAB_WAKE_QY: WAKE_DIRS,
                 TAB_CARRY: nb * 2}
        n = sizes.get(table, nb)
        out = np.zeros(n, dtype=_TABLE_DTYPES[table])
        _check(lib().scwp_get_table(self.ctx, p, table, out.ctypes.data_as(C.c_void_p),
                                    out.nbytes), self.ctx)
        return out

    def particles(self, p=0):
        info = self.info(p)
        cap = info.capacity
        x = np.zeros(cap, np.int32)
        y = np.zeros(cap, np.int32)
        bd = np.zeros(cap, np.uint32)
        n = C.c_int64()
        _check(lib().scwp_get_particles(self.ctx, p, x.ctypes.data_as(C.c_void_p),
                                        y.ctypes.data_as(C.c_void_p),
                                        bd.ctypes.data_as(C.c_void_p), cap, C.byref(n)), self.ctx)
        k = n.value
        return x[:k].copy(), y[:k].copy(), bd[:k].copy()

    def set_particles(self, p, x, y, bd):
        x = np.ascontiguousarray(x, np.int32)
        y = np.ascontiguousarray(y, np.int32)
        bd = np.ascontiguousarray(bd, np.uint32)
        _check(lib().scwp_set_particles(self.ctx, p, x.ctypes.data_as(C.c_void_p),
                                        y.ctypes.data_as(C.c_void_p),
                                        bd.ctypes.data_as(C.c_void_p), len(x)), self.ctx)

    def bins(self, p=0):
        info = self.info(p)
        tb = info.total_bins
        counts = np.zeros(tb, np.uint32)
        offsets = np.zeros(tb + 1, np.uint32)
        n = C.c_int64()
        _check(lib().scwp_get_bins(self.ctx, p, counts.ctypes.data_as(C.c_void_p),
                                   offsets.ctypes.data_as(C.c_void_p), None, 0, C.byref(n)),
               self.ctx)
        entries = np.zeros(max(n.value, 1), np.uint32)
        _check(lib().scwp_get_bins(self.ctx, p, None, None, entries.ctypes.data_as(C.c_void_p),
                                   len(entries), C.byref(n)), self.ctx)
        return counts, offsets, entries[:n.value]

    def resynthesize(self, mode=SYNTH_SAT):
        _check(lib().scwp_resynthesize(self.ctx, mode), self.ctx)

    def set_synth_mode(self, mode):
        _check(lib().scwp_set_synth_mode(self.ctx, mode), self.ctx)

    def set_sat_plan(self, variant, gmul=1.0):
        _check(lib().scwp_set_sat_plan(self.ctx, int(variant), float(gmul)), self.ctx)

    def autotune(self, reps=3, force=False):
        """scwp_autotune: time the summed-area variants and bucket-group
        multipliers on the last frame and keep the fastest; returns the
        table [(variant, gmul, ms)], the chosen index and whether the choice
        came from the per-device cache."""
        r = scwp_tune_result()
        _check(lib().scwp_autotune(self.ctx, int(reps), 1 if force else 0, C.byref(r)), self.ctx)
        rows = [(int(r.variant[k]), float(r.gmul[k]), float(r.ms[k])) for k in range(r.n_configs)]
        return rows, int(r.chosen), bool(r.from_cache)

    def set_batched(self, on):
        _check(lib().scwp_set_batched(self.ctx, 1 if on else 0), self.ctx)

    def normals(self, p):
        """Unit normals (nx, ny, nz) of patch p's last blended maps, float32 [3, H, W]."""
        H, W = self.patch_shape(p)
        a = np.empty((3, H, W), dtype=np.float32)
        _check(lib().scwp_normal_map(self.ctx, int(p), a.ctypes.data_as(C.c_void_p), a.size, 0), self.ctx)
        return a

    def set_bucket_range(self, b_lo, b_hi):
        _check(lib().scwp_set_bucket_range(self.ctx, int(b_lo), int(b_hi)), self.ctx)

    def set_timing(self, on):
        _check(lib().scwp_set_timing(self.ctx, 1 if on else 0), self.ctx)

    def launch_count(self):
        n = C.c_int64()
        _check(lib().scwp_launch_count(self.ctx, C.byref(n)), self.ctx)
        return n.value

    def timing_read(self):
        ms = (C.c_double * 4)()
        fr = C.c_int64()
        _check(lib().scwp_timing_read(self.ctx, ms, C.byref(fr)), self.ctx)
        return list(ms), fr.value


class _ServerSceneView(Scene):
    """A server scene's context, read like a Scene (maps, stats, info);
    the server owns and releases it."""

    def __init__(self, ctx, cfg, device):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.device = device
        self.ctx = ctx
        self.N = int(cfg["spectrum"]["fft_n"])

    def close(self):
        self.ctx = None


class Server:
    """The frame-step server of the C ABI (scwp_server_*): scenes admitted
    against a device-memory budget, requests batched into ticks."""

    def __init__(self, hbm_budget_bytes=0, max_inflight=3, device=0, stream=None, use_torch_alloc=True):
        import torch
        self.device = device
        torch.cuda.set_device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._alloc = self._free = None
        if use_torch_alloc:
            st = self.stream

            def _a(nbytes, user):
                try:
                    return int(torch.cuda.caching_allocator_alloc(int(nbytes), device, st))
                except Exception:
                    return None

            def _f(ptr, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._alloc = ALLOC_FN(_a)
            self._free = FREE_FN(_f)
        d = scwp_server_desc()
        d.stream = C.c_void_p(self.stream.cuda_stream)
        d.hbm_budget_bytes = int(hbm_budget_bytes)
        d.max_inflight = int(max_inflight)
        if self._alloc is not None:
            d.alloc = self._alloc
            d.free = self._free
        self.sv = C.c_void_p()
        self._check(lib().scwp_server_create(C.byref(d), C.byref(self.sv)))
        self.cfgs = {}
        self._ids = (C.c_int64 * 65536)()

    def _check(self, status):
        if status != 0:
            msg = lib().scwp_server_last_error(self.sv).decode() if getattr(self, "sv", None) else ""
            raise ScwpError(status, msg)

    def close(self):
        if getattr(self, "sv", None):
            lib().scwp_server_destroy(self.sv)
            self.sv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_scene(self, cfg):
        """Admit a scene; its id, or None when the memory budget refuses it."""
        sd = spectrum_desc(cfg["spectrum"])
        arr = (scwp_patch_desc * len(cfg["patches"]))(*[patch_desc(p) for p in cfg["patches"]])
        sid = C.c_int32()
        rc = lib().scwp_server_add_scene(self.sv, C.byref(sd), C.cast(arr, C.c_void_p), len(cfg["patches"]),
                                         C.byref(sid))
        if rc == 2:
            return None
        self._check(rc)
        self.cfgs[sid.value] = cfg
        return sid.value

    def remove_scene(self, sid):
        self._check(lib().scwp_server_remove_scene(self.sv, int(sid)))
        self.cfgs.pop(int(sid), None)

    def submit(self, sid, dt, request_id):
        self._check(lib().scwp_server_submit(self.sv, int(sid), float(dt), int(request_id)))

    def tick(self):
        n = C.c_int32()
        self._check(lib().scwp_server_tick(self.sv, C.byref(n)))
        return n.value

    def poll(self):
        n = C.c_int32()
        self._check(lib().scwp_server_poll(self.sv, C.cast(self._ids, C.c_void_p), len(self._ids), C.byref(n)))
        return [self._ids[k] for k in range(n.value)]

    def scene(self, sid):
        c = C.c_void_p()
        self._check(lib().scwp_server_scene(self.sv, int(sid), C.byref(c)))
        return _ServerSceneView(c, self.cfgs[int(sid)], self.device)

    def info(self):
        out = scwp_server_info()
        self._check(lib().scwp_server_info_get(self.sv, C.byref(out)))
        return out
