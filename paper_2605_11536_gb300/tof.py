"""Thin ctypes binding of libtof.so (include/tof.h): the same entry points, argument
marshalling only.  Every step of the rendering path runs in the library's CUDA kernels; there is
no Python or CPU fallback -- loading fails loudly when the library or a GPU is missing.

Device buffers are passed as raw pointers (``tensor.data_ptr()``) and streams as
``torch.cuda.Stream.cuda_stream`` integers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None


class TofError(RuntimeError):
    pass


class tof_material(C.Structure):
    _fields_ = [("type", C.c_int32), ("albedo", C.c_float), ("alpha", C.c_float)]


class tof_sensor(C.Structure):
    _fields_ = [("mode", C.c_int32), ("W", C.c_int32), ("H", C.c_int32), ("pos", C.c_float * 3),
                ("fwd", C.c_float * 3), ("up", C.c_float * 3), ("fov_y", C.c_float), ("wall_o", C.c_float * 3),
                ("wall_u", C.c_float * 3), ("wall_v", C.c_float * 3)]


class tof_emitter(C.Structure):
    _fields_ = [("type", C.c_int32), ("pos", C.c_float * 3), ("dir", C.c_float * 3), ("power", C.c_float)]


class tof_gate(C.Structure):
    _fields_ = [("L0", C.c_float), ("dL", C.c_float)]


class tof_bins(C.Structure):
    _fields_ = [("t0", C.c_float), ("width", C.c_float), ("B", C.c_int32)]


class tof_params(C.Structure):
    _fields_ = [("depth", C.c_int32), ("n_cand", C.c_int32), ("n_spatial", C.c_int32), ("radius", C.c_int32),
                ("n_spatial_iters", C.c_int32), ("temporal", C.c_int32), ("m_cap", C.c_float),
                ("newton_max_iter", C.c_int32), ("newton_tol_frac", C.c_float), ("jac_max", C.c_float),
                ("d_min", C.c_float), ("ray_eps", C.c_float), ("flags", C.c_uint32), ("shrink_k", C.c_float),
                ("shrink_fine", C.c_int32)]


class tof_job(C.Structure):
    pass


class tof_tuning(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("packet", C.c_int32), ("layout", C.c_int32)]


LAYOUT_SOA, LAYOUT_AOS = 0, 1


EXPORTS = ["tof_create", "tof_destroy", "tof_last_error", "tof_device_bytes", "tof_scene_upload", "tof_scene_destroy",
           "tof_bvh_build", "tof_view_create", "tof_view_destroy", "tof_render_gated", "tof_render_transient",
           "tof_render_pt", "tof_reservoirs_reset", "tof_view_stats", "tof_view_profile", "tof_view_stage_ms",
           "tof_render_gated_noalloc", "tof_render_batch", "tof_server_create", "tof_server_destroy",
           "tof_server_open_stream", "tof_server_submit", "tof_server_step", "tof_server_poll", "tof_server_stats",
           "tof_view_set_tuning", "tof_view_get_tuning", "tof_autotune", "tof_sync", "tof_kernel_launches"]

_vp, _fp, _u32p = C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_uint32)

tof_job._fields_ = [("scene", C.c_int32), ("view", C.c_int32), ("sensor", tof_sensor), ("emitter", tof_emitter),
                    ("gate", tof_gate), ("bins", tof_bins), ("transient", C.c_int32), ("params", tof_params),
                    ("seed", C.c_uint64), ("frame", C.c_uint32), ("out_dev", C.c_void_p)]


def _declare(L):
    L.tof_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_uint64]
    L.tof_destroy.argtypes = [_vp]
    L.tof_last_error.argtypes = [_vp]
    L.tof_last_error.restype = C.c_char_p
    L.tof_device_bytes.argtypes = [_vp]
    L.tof_device_bytes.restype = C.c_uint64
    L.tof_scene_upload.argtypes = [_vp, _fp, C.c_uint32, _u32p, C.c_uint32, _u32p, C.POINTER(tof_material), C.c_uint32,
                                   _u32p, C.c_uint32, C.POINTER(C.c_int32)]
    L.tof_scene_destroy.argtypes = [_vp, C.c_int32]
    L.tof_bvh_build.argtypes = [_vp, C.c_int32, _fp, C.c_int, _vp]
    L.tof_view_create.argtypes = [_vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]
    L.tof_view_destroy.argtypes = [_vp, C.c_int32]
    L.tof_render_gated.argtypes = [_vp, C.c_int32, C.c_int32, C.POINTER(tof_sensor), C.POINTER(tof_emitter),
                                   C.POINTER(tof_gate), C.POINTER(tof_params), C.c_uint64, C.c_uint32, _vp, _vp]
    L.tof_render_gated_noalloc.argtypes = [_vp, C.c_int32, C.c_int32, C.POINTER(tof_sensor), C.POINTER(tof_emitter),
                                           C.POINTER(tof_gate), C.POINTER(tof_params), C.c_uint64, C.c_uint32, _vp, _vp]
    L.tof_render_transient.argtypes = [_vp, C.c_int32, C.c_int32, C.POINTER(tof_sensor), C.POINTER(tof_emitter),
                                       C.POINTER(tof_bins), C.POINTER(tof_params), C.c_uint64, C.c_uint32, _vp, _vp]
    L.tof_render_pt.argtypes = [_vp, C.c_int32, C.POINTER(tof_sensor), C.POINTER(tof_emitter), C.POINTER(tof_gate),
                                C.POINTER(tof_bins), C.POINTER(tof_params), C.c_uint64, C.c_uint32, C.c_int32, _vp, _vp]
    L.tof_reservoirs_reset.argtypes = [_vp, C.c_int32]
    L.tof_render_batch.argtypes = [_vp, C.POINTER(tof_job), C.c_uint32, _vp]
    L.tof_view_set_tuning.argtypes = [_vp, C.c_int32, C.POINTER(tof_tuning)]
    L.tof_view_get_tuning.argtypes = [_vp, C.c_int32, C.POINTER(tof_tuning)]
    L.tof_autotune.argtypes = [_vp, C.POINTER(tof_job), C.c_uint32, C.c_int32, _vp, C.POINTER(tof_tuning)]
    L.tof_server_create.argtypes = [_vp, C.c_uint64, C.POINTER(C.c_void_p)]
    L.tof_server_destroy.argtypes = [_vp]
    L.tof_server_open_stream.argtypes = [_vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]
    L.tof_server_submit.argtypes = [_vp, C.c_int32, C.POINTER(tof_job), _fp, C.POINTER(C.c_uint64)]
    L.tof_server_step.argtypes = [_vp, _vp]
    L.tof_server_poll.argtypes = [_vp, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    L.tof_server_stats.argtypes = [_vp, C.POINTER(C.c_double)]
    L.tof_view_stats.argtypes = [_vp, C.c_int32, C.POINTER(C.c_double)]
    L.tof_view_profile.argtypes = [_vp, C.c_int32, C.c_int]
    L.tof_view_stage_ms.argtypes = [_vp, C.c_int32, C.POINTER(C.c_float)]
    L.tof_sync.argtypes = [_vp, _vp]
    L.tof_kernel_launches.argtypes = []
    L.tof_kernel_launches.restype = C.c_uint64
    for name in EXPORTS:
        if name not in ("tof_last_error", "tof_device_bytes", "tof_kernel_launches"):
            getattr(L, name).restype = C.c_int32


def lib(build: bool = True):
    """Load libtof.so (building it first when stale).  Raises if it cannot be built or loaded."""
    global _LIB
    if _LIB is None:
        path = _build.build() if build else _build.OUT
        if not os.path.exists(path):
            raise TofError("libtof.so is missing (%s); run paper_2605_11536_gb300.build.build()" % path)
        _LIB = C.CDLL(path)
        _declare(_LIB)
    return _LIB


def library_path() -> str:
    return _build.OUT


# ---------------------------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------------------------
def sensor(d: dict) -> tof_sensor:
    s = tof_sensor()
    s.mode, s.W, s.H = int(d["mode"]), int(d["W"]), int(d["H"])
    for f in ("pos", "fwd", "up", "wall_o", "wall_u", "wall_v"):
        getattr(s, f)[:] = [float(x) for x in d.get(f, [0.0, 0.0, 0.0])]
    s.fov_y = float(d.get("fov_y", 0.0))
    return s


def emitter(d: dict) -> tof_emitter:
    e = tof_emitter()
    e.type = int(d["type"])
    e.pos[:] = [float(x) for x in d["pos"]]
    e.dir[:] = [float(x) for x in d.get("dir", [0, 0, -1])]
    e.power = float(d["power"])
    return e


def params(p) -> tof_params:
    o = tof_params()
    for name, _ in tof_params._fields_:
        setattr(o, name, getattr(p, name))
    return o


def _check(ctx, rc, what):
    if rc != 0:
        msg = lib().tof_last_error(ctx).decode() if ctx else ""
        raise TofError("%s failed (status %d): %s" % (what, rc, msg))


# ---------------------------------------------------------------------------------------------
# entry points (same names as include/tof.h)
# ---------------------------------------------------------------------------------------------
def tof_create(device: int = 0, hbm_budget_bytes: int = 0):
    ctx = C.c_void_p()
    rc = lib().tof_create(C.byref(ctx), device, hbm_budget_bytes)
    if rc != 0:
        raise TofError("tof_create failed (status %d): no usable CUDA device %d" % (rc, device))
    return ctx


def tof_destroy(ctx):
    _check(None, lib().tof_destroy(ctx), "tof_destroy")


def tof_last_error(ctx) -> str:
    return lib().tof_last_error(ctx).decode()


def tof_device_bytes(ctx) -> int:
    return int(lib().tof_device_bytes(ctx))


def tof_scene_upload(ctx, verts, tris, tri_object, materials, object_material) -> int:
    v = np.ascontiguousarray(verts, dtype=np.float32)
    t = np.ascontiguousarray(tris, dtype=np.uint32)
    to = np.ascontiguousarray(tri_object, dtype=np.uint32)
    om = np.ascontiguousarray(object_material, dtype=np.uint32)
    mats = np.asarray(materials, dtype=np.float64)
    M = (tof_material * len(mats))()
    for i, (ty, al, a) in enumerate(mats):
        M[i].type, M[i].albedo, M[i].alpha = int(ty), float(al), float(a)
    out = C.c_int32()
    rc = lib().tof_scene_upload(ctx, v.ctypes.data_as(_fp), len(v), t.ctypes.data_as(_u32p), len(t),
                                to.ctypes.data_as(_u32p), M, len(mats), om.ctypes.data_as(_u32p), len(om), C.byref(out))
    _check(ctx, rc, "tof_scene_upload")
    return out.value


def tof_scene_destroy(ctx, scene: int):
    _check(ctx, lib().tof_scene_destroy(ctx, scene), "tof_scene_destroy")


def tof_bvh_build(ctx, scene: int, object_xforms, refit_only: int = 0, stream: int = 0):
    x = np.ascontiguousarray(object_xforms, dtype=np.float32)
    _check(ctx, lib().tof_bvh_build(ctx, scene, x.ctypes.data_as(_fp), int(refit_only), C.c_void_p(stream)), "tof_bvh_build")


def tof_view_create(ctx, scene: int, W: int, H: int, B: int = 0) -> int:
    out = C.c_int32()
    _check(ctx, lib().tof_view_create(ctx, scene, W, H, B, C.byref(out)), "tof_view_create")
    return out.value


def tof_view_destroy(ctx, view: int):
    _check(ctx, lib().tof_view_destroy(ctx, view), "tof_view_destroy")


def tof_render_gated(ctx, scene, view, sensor_d, emitter_d, gate, params_p, seed, frame, out_ptr, stream=0):
    s, e, p = sensor(sensor_d), emitter(emitter_d), params(params_p)
    g = tof_gate(float(gate[0]), float(gate[1]))
    rc = lib().tof_render_gated(ctx, scene, view, C.byref(s), C.byref(e), C.byref(g), C.byref(p), int(seed), int(frame),
                                C.c_void_p(out_ptr), C.c_void_p(stream))
    _check(ctx, rc, "tof_render_gated")


def tof_render_gated_noalloc(ctx, scene, view, sensor_d, emitter_d, gate, params_p, seed, frame, out_ptr, stream=0):
    """tof_render_gated without device allocation inside the call (static reuse scratch; see tof.h)."""
    s, e, p = sensor(sensor_d), emitter(emitter_d), params(params_p)
    g = tof_gate(float(gate[0]), float(gate[1]))
    rc = lib().tof_render_gated_noalloc(ctx, scene, view, C.byref(s), C.byref(e), C.byref(g), C.byref(p), int(seed),
                                        int(frame), C.c_void_p(out_ptr), C.c_void_p(stream))
    _check(ctx, rc, "tof_render_gated_noalloc")


def tof_render_transient(ctx, scene, view, sensor_d, emitter_d, bins, params_p, seed, frame, out_ptr, stream=0):
    s, e, p = sensor(sensor_d), emitter(emitter_d), params(params_p)
    b = tof_bins(float(bins[0]), float(bins[1]), int(bins[2]))
    rc = lib().tof_render_transient(ctx, scene, view, C.byref(s), C.byref(e), C.byref(b), C.byref(p), int(seed),
                                    int(frame), C.c_void_p(out_ptr), C.c_void_p(stream))
    _check(ctx, rc, "tof_render_transient")


def tof_render_pt(ctx, scene, sensor_d, emitter_d, gate, bins, params_p, seed, frame, spp, out_ptr, stream=0):
    s, e, p = sensor(sensor_d), emitter(emitter_d), params(params_p)
    g = tof_gate(float(gate[0]), float(gate[1])) if gate is not None else None
    b = tof_bins(float(bins[0]), float(bins[1]), int(bins[2])) if bins is not None else None
    rc = lib().tof_render_pt(ctx, scene, C.byref(s), C.byref(e), C.byref(g) if g else None, C.byref(b) if b else None,
                             C.byref(p), int(seed), int(frame), int(spp), C.c_void_p(out_ptr), C.c_void_p(stream))
    _check(ctx, rc, "tof_render_pt")


def tof_sync(ctx, stream: int = 0):
    """Wait for `stream`; raises TofError if a kernel recorded a device-side error since the last check."""
    _check(ctx, lib().tof_sync(ctx, C.c_void_p(stream)), "tof_sync")


def tof_kernel_launches() -> int:
    return int(lib().tof_kernel_launches())


def tof_reservoirs_reset(ctx, view: int):
    _check(ctx, lib().tof_reservoirs_reset(ctx, view), "tof_reservoirs_reset")


def tof_view_stats(ctx, view: int):
    a = (C.c_double * 10)()
    _check(ctx, lib().tof_view_stats(ctx, view, a), "tof_view_stats")
    return dict(newton_calls=a[0], newton_iters=a[1], newton_ok=a[2], shift_calls=a[3], shift_ok=a[4], inv_calls=a[5],
                spatial_fwd_calls=a[6], spatial_inv_calls=a[7], spatial_fwd_rays=a[8], spatial_inv_rays=a[9])


def tof_view_profile(ctx, view: int, enable: int = 1):
    _check(ctx, lib().tof_view_profile(ctx, view, int(enable)), "tof_view_profile")


STAGES = ("gbuffer", "initial", "temporal", "spatial", "splat", "frame", "spatial_setup", "spatial_fwd_shift",
          "spatial_inv_shift", "spatial_merge", "spatial_fwd_vis", "spatial_inv_vis")


def tof_view_stage_ms(ctx, view: int):
    a = (C.c_float * 12)()
    _check(ctx, lib().tof_view_stage_ms(ctx, view, a), "tof_view_stage_ms")
    return dict(zip(STAGES, [float(x) for x in a]))


def job(scene, view, sensor_d, emitter_d, params_p, seed, frame, out_ptr, gate=None, bins=None) -> tof_job:
    j = tof_job()
    j.scene, j.view = int(scene), int(view)
    j.sensor, j.emitter, j.params = sensor(sensor_d), emitter(emitter_d), params(params_p)
    if bins is not None:
        j.bins = tof_bins(float(bins[0]), float(bins[1]), int(bins[2]))
        j.transient = 1
    else:
        j.gate = tof_gate(float(gate[0]), float(gate[1]))
        j.transient = 0
    j.seed, j.frame, j.out_dev = int(seed), int(frame), int(out_ptr)
    return j


def tof_render_batch(ctx, jobs, stream: int = 0):
    arr = (tof_job * len(jobs))(*jobs)
    _check(ctx, lib().tof_render_batch(ctx, arr, len(jobs), C.c_void_p(stream)), "tof_render_batch")


def tof_view_set_tuning(ctx, view: int, tile_w: int = 16, tile_h: int = 8, packet: int = 0, layout: int = LAYOUT_SOA):
    t = tof_tuning(int(tile_w), int(tile_h), int(packet), int(layout))
    _check(ctx, lib().tof_view_set_tuning(ctx, view, C.byref(t)), "tof_view_set_tuning")


def tof_view_get_tuning(ctx, view: int) -> dict:
    t = tof_tuning()
    _check(ctx, lib().tof_view_get_tuning(ctx, view, C.byref(t)), "tof_view_get_tuning")
    return dict(tile_w=t.tile_w, tile_h=t.tile_h, packet=t.packet, layout=t.layout)


def tof_autotune(ctx, jobs, frames: int = 3, stream: int = 0):
    """Tune every job's view (tof_autotune); returns each job's chosen tuning as a dict."""
    arr = (tof_job * len(jobs))(*jobs)
    out = (tof_tuning * len(jobs))()
    _check(ctx, lib().tof_autotune(ctx, arr, len(jobs), int(frames), C.c_void_p(stream), out), "tof_autotune")
    return [dict(tile_w=t.tile_w, tile_h=t.tile_h, packet=t.packet, layout=t.layout) for t in out]


def tof_server_create(ctx, hbm_budget_bytes: int = 0):
    s = C.c_void_p()
    _check(ctx, lib().tof_server_create(ctx, int(hbm_budget_bytes), C.byref(s)), "tof_server_create")
    return s


def tof_server_destroy(srv):
    _check(None, lib().tof_server_destroy(srv), "tof_server_destroy")


def tof_server_open_stream(srv, scene: int, W: int, H: int, B: int = 0) -> int:
    out = C.c_int32()
    _check(None, lib().tof_server_open_stream(srv, scene, W, H, B, C.byref(out)), "tof_server_open_stream")
    return out.value


def tof_server_submit(srv, stream_id: int, job_s: tof_job, object_xforms) -> int:
    x = np.ascontiguousarray(object_xforms, dtype=np.float32)
    t = C.c_uint64()
    _check(None, lib().tof_server_submit(srv, stream_id, C.byref(job_s), x.ctypes.data_as(_fp), C.byref(t)),
           "tof_server_submit")
    return t.value


def tof_server_step(srv, stream: int = 0):
    _check(None, lib().tof_server_step(srv, C.c_void_p(stream)), "tof_server_step")


def tof_server_poll(srv, ticket: int):
    st, lat = C.c_int32(), C.c_double()
    _check(None, lib().tof_server_poll(srv, int(ticket), C.byref(st), C.byref(lat)), "tof_server_poll")
    return st.value, lat.value


def tof_server_stats(srv):
    a = (C.c_double * 7)()
    _check(None, lib().tof_server_stats(srv, a), "tof_server_stats")
    return dict(submitted=a[0], completed=a[1], batches=a[2], deferred=a[3], resident_bytes=a[4], queued=a[5],
                inflight=a[6])
