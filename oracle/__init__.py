"""CPU oracle of the ToF ReSTIR hot path (FP64, plain C) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import this package.  The product path (``paper_2605_11536_gb300``) never
imports it and shares no code with it.

``build()`` compiles ``tof_oracle.c`` into ``liboracle.so`` next to this file with gcc.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tof_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        # no fused multiply-add contraction: the same FP64 rounding on every host architecture
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        _declare(_lib)
    return _lib


class OSensor(C.Structure):
    _fields_ = [("mode", C.c_int), ("W", C.c_int), ("H", C.c_int), ("pos", C.c_double * 3),
                ("fwd", C.c_double * 3), ("up", C.c_double * 3), ("fov_y", C.c_double),
                ("wall_o", C.c_double * 3), ("wall_u", C.c_double * 3), ("wall_v", C.c_double * 3)]


class OEmitter(C.Structure):
    _fields_ = [("type", C.c_int), ("pos", C.c_double * 3), ("dir", C.c_double * 3), ("power", C.c_double)]


class OParams(C.Structure):
    _fields_ = [("depth", C.c_int), ("n_cand", C.c_int), ("n_spatial", C.c_int), ("radius", C.c_int),
                ("n_spatial_iters", C.c_int), ("temporal", C.c_int), ("m_cap", C.c_double),
                ("newton_max_iter", C.c_int), ("newton_tol_frac", C.c_double), ("jac_max", C.c_double),
                ("d_min", C.c_double), ("ray_eps", C.c_double), ("flags", C.c_uint32), ("shrink_k", C.c_double),
                ("shrink_fine", C.c_int)]


_dp = C.POINTER(C.c_double)
_u32p = C.POINTER(C.c_uint32)


def _declare(L):
    L.or_philox.argtypes = [_u32p, _u32p, _u32p]
    L.or_geom_create.restype = C.c_void_p
    L.or_geom_create.argtypes = [_dp, C.c_int, _u32p, C.c_int, _u32p, _u32p, C.c_int, _dp, C.c_int, _dp]
    L.or_geom_destroy.argtypes = [C.c_void_p]
    L.or_geom_intersect.restype = C.c_int
    L.or_geom_intersect.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_int, _dp, C.POINTER(C.c_int), _dp, _dp]
    L.or_view_create.restype = C.c_void_p
    L.or_view_create.argtypes = [C.c_int, C.c_int, C.c_int]
    L.or_view_destroy.argtypes = [C.c_void_p]
    L.or_view_reset.argtypes = [C.c_void_p]
    L.or_view_stats.argtypes = [C.c_void_p, _dp]
    L.or_render_frame.restype = C.c_int
    L.or_render_frame.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(OSensor), C.POINTER(OEmitter), C.c_double,
                                  C.c_double, C.c_int, C.POINTER(OParams), C.c_uint64, C.c_uint32, C.c_int,
                                  C.c_int, C.c_int, C.c_int, _dp, C.POINTER(C.c_uint8), C.c_int]
    L.or_render_pt.restype = C.c_int
    L.or_render_pt.argtypes = [C.c_void_p, C.POINTER(OSensor), C.POINTER(OEmitter), C.c_double, C.c_double,
                               C.c_int, C.POINTER(OParams), C.c_uint64, C.c_uint32, C.c_int, C.c_int, C.c_int,
                               C.c_int, C.c_int, _dp, C.c_int]
    L.or_bsdf_eval.restype = C.c_double
    L.or_bsdf_eval.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _dp]
    L.or_bsdf_pdf.restype = C.c_double
    L.or_bsdf_pdf.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _dp]
    L.or_bsdf_sample.restype = C.c_int
    L.or_bsdf_sample.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, C.c_double, C.c_double, _dp, _dp, _dp]
    L.or_length_derivs.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.or_newton.restype = C.c_int
    L.or_newton.argtypes = [_dp] * 10 + [_dp, C.c_double, C.c_int, C.c_double, C.c_double, _dp, _dp,
                                         C.POINTER(C.c_int), _dp]
    L.or_newton_g.restype = C.c_int
    L.or_newton_g.argtypes = [_dp] * 10 + [_dp, C.c_double, C.c_int, C.c_double, C.c_double, _dp, _dp,
                                           C.POINTER(C.c_int), _dp, C.c_int]
    L.or_stream_select.restype = C.c_int
    L.or_stream_select.argtypes = [_dp, _dp, C.c_int, _dp]
    L.or_ris_accept.restype = C.c_int
    L.or_ris_accept.argtypes = [C.c_double, C.c_double, C.c_double, _dp]
    L.or_ris_W.restype = C.c_double
    L.or_ris_W.argtypes = [C.c_double, C.c_double]
    L.or_gris_mis.restype = C.c_double
    L.or_gris_mis.argtypes = [_dp, _dp, C.c_int, C.c_int, C.c_int]
    L.or_view_reservoir.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp, C.POINTER(C.c_int)]
    L.or_shift_roundtrip.restype = C.c_int
    L.or_shift_roundtrip.argtypes = [C.c_void_p, C.POINTER(OParams), C.c_uint64, C.c_int, C.c_int, _dp]
    L.or_shrink_roundtrip.restype = C.c_int
    L.or_shrink_roundtrip.argtypes = [C.c_void_p, C.POINTER(OParams), C.c_uint64, C.c_int, C.c_double, _dp]
    L.or_ell_sample.restype = C.c_int
    L.or_ell_sample.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_double, _u32p, _dp]
    L.or_ell_pdf.restype = C.c_double
    L.or_ell_pdf.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_double, C.c_int, C.c_double, C.c_double]
    L.or_ell_tri_probs.argtypes = [C.c_void_p, _dp, _dp, C.c_double, _dp]


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _u(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a, a.ctypes.data_as(_u32p)


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox(c, k, o)
    return [int(x) for x in o]


def sensor_struct(s: dict) -> OSensor:
    o = OSensor()
    o.mode, o.W, o.H = int(s["mode"]), int(s["W"]), int(s["H"])
    for f in ("pos", "fwd", "up", "wall_o", "wall_u", "wall_v"):
        getattr(o, f)[:] = [float(x) for x in s.get(f, [0.0, 0.0, 0.0])]
    o.fov_y = float(s.get("fov_y", 0.0))
    return o


def emitter_struct(e: dict) -> OEmitter:
    o = OEmitter()
    o.type = int(e["type"])
    o.pos[:] = [float(x) for x in e["pos"]]
    o.dir[:] = [float(x) for x in e.get("dir", [0, 0, -1])]
    o.power = float(e["power"])
    return o


def params_struct(p) -> OParams:
    o = OParams()
    for name, _ in OParams._fields_:
        setattr(o, name, getattr(p, name))
    return o


class Geom:
    """World-space geometry of one frame (transformed triangles + the oracle's own BVH)."""

    def __init__(self, scene, frame: int = 0, xforms=None):
        L = lib()
        xf = scene.xforms[frame] if xforms is None else xforms
        self._keep = [_d(scene.verts), _u(scene.tris), _u(scene.tri_object), _u(scene.object_material),
                      _d(scene.materials), _d(xf)]
        (v, vp), (t, tp), (to, top), (om, omp), (m, mp), (x, xp) = self._keep
        self.ptr = L.or_geom_create(vp, len(v), tp, len(t), top, omp, len(om), mp, len(m), xp)

    def intersect(self, o, d, tmax=1e30, brute=False):
        L = lib()
        (oo, op), (dd, dp) = _d(o), _d(d)
        t, b1, b2 = C.c_double(), C.c_double(), C.c_double()
        tri = C.c_int()
        hit = L.or_geom_intersect(self.ptr, op, dp, tmax, int(brute), C.byref(t), C.byref(tri), C.byref(b1), C.byref(b2))
        return (tri.value, t.value, b1.value, b2.value) if hit else None

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.or_geom_destroy(self.ptr)
            self.ptr = None


class View:
    """Per-view state across frames (current / previous G-buffers and reservoirs)."""

    def __init__(self, W: int, H: int, B: int = 0):
        self.W, self.H, self.B = W, H, B
        self.ptr = lib().or_view_create(W, H, B)

    def reset(self):
        lib().or_view_reset(self.ptr)

    def stats(self):
        a = np.zeros(5)
        lib().or_view_stats(self.ptr, a.ctypes.data_as(_dp))
        return dict(newton_calls=a[0], newton_iters=a[1], newton_ok=a[2], shift_calls=a[3], shift_ok=a[4])

    def reservoir(self, pix: int, b: int = 0):
        out = np.zeros(4)
        iout = (C.c_int * 3)()
        lib().or_view_reservoir(self.ptr, pix, b, out.ctypes.data_as(_dp), iout)
        return dict(W=out[0], M=out[1], phat=out[2], tau=out[3], k=iout[0], r=iout[1], valid=iout[2])

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.or_view_destroy(self.ptr)
            self.ptr = None


def render_frame(view: View, geom: Geom, scene, frame: int, params=None, seed=None, roi=None, nthreads=0,
                 frame_index=None):
    """One frame of the pipeline; returns (image [H, W] or histogram [H, W, B], ok mask [H, W])."""
    p = params if params is not None else scene.params
    s = sensor_struct(scene.sensors[frame])
    e = emitter_struct(scene.emitters[frame])
    if scene.bins is not None and view.B > 0:
        L0, dL, B = scene.bins[0], scene.bins[1], view.B
    else:
        (L0, dL), B = scene.gates[frame], 0
    W, H = view.W, view.H
    Bn = B if B > 0 else 1
    out = np.zeros(W * H * Bn)
    ok = np.zeros(W * H, dtype=np.uint8)
    x0, y0, x1, y1 = roi if roi is not None else (0, 0, W, H)
    pp = params_struct(p)
    rc = lib().or_render_frame(view.ptr, geom.ptr, C.byref(s), C.byref(e), L0, dL, B, C.byref(pp),
                               scene.seed if seed is None else seed, frame if frame_index is None else frame_index,
                               x0, y0, x1, y1, out.ctypes.data_as(_dp), ok.ctypes.data_as(C.POINTER(C.c_uint8)),
                               nthreads)
    if rc != 0:
        raise ValueError("oracle rejected the frame arguments")
    img = out.reshape(H, W, Bn) if B > 0 else out.reshape(H, W)
    return img, ok.reshape(H, W).astype(bool)


def render_pt(geom: Geom, scene, frame: int, spp: int, params=None, seed=None, roi=None, nthreads=0, B=0):
    p = params if params is not None else scene.params
    s = sensor_struct(scene.sensors[frame])
    e = emitter_struct(scene.emitters[frame])
    if B > 0:
        L0, dL = scene.bins[0], scene.bins[1]
    else:
        L0, dL = scene.gates[frame]
    W, H = int(scene.sensors[frame]["W"]), int(scene.sensors[frame]["H"])
    Bn = B if B > 0 else 1
    out = np.zeros(W * H * Bn)
    x0, y0, x1, y1 = roi if roi is not None else (0, 0, W, H)
    pp = params_struct(p)
    lib().or_render_pt(geom.ptr, C.byref(s), C.byref(e), L0, dL, B, C.byref(pp),
                       scene.seed if seed is None else seed, frame, spp, x0, y0, x1, y1,
                       out.ctypes.data_as(_dp), nthreads)
    return out.reshape(H, W, Bn) if B > 0 else out.reshape(H, W)


def bsdf_eval(type_, albedo, alpha, n, wi, wo):
    return lib().or_bsdf_eval(type_, albedo, alpha, _d(n)[1], _d(wi)[1], _d(wo)[1])


def bsdf_pdf(type_, albedo, alpha, n, wi, wo):
    return lib().or_bsdf_pdf(type_, albedo, alpha, _d(n)[1], _d(wi)[1], _d(wo)[1])


def bsdf_sample(type_, albedo, alpha, n, wi, u0, u1):
    wo = np.zeros(3)
    pdf, thr = C.c_double(), C.c_double()
    a, ap = _d(n)
    b, bp = _d(wi)
    ok = lib().or_bsdf_sample(type_, albedo, alpha, ap, bp, u0, u1, wo.ctypes.data_as(_dp), C.byref(pdf), C.byref(thr))
    return bool(ok), wo, pdf.value, thr.value


def length_derivs(p1, p2, o, t, b, xi):
    L, g, h = C.c_double(), np.zeros(2), np.zeros(3)
    args = [_d(p1), _d(p2), _d(o), _d(t), _d(b), _d(xi)]
    lib().or_length_derivs(*[a[1] for a in args], C.byref(L), g.ctypes.data_as(_dp), h.ctypes.data_as(_dp))
    return L.value, g, h


GAUGES = {"average": 0, "axis_t": 1, "axis_b": 2, "start": 3}


def newton(base, offset, xi, delta, max_iter=5, tol_stop=1e-12, tol_succ=1e-9, gauge="average"):
    """base / offset: dict(p1, p2, o, t, b) of the two paths.  Returns (ok, xi', |det|, iters, F)."""
    arrs = [_d(base[k]) for k in ("p1", "p2", "o", "t", "b")] + [_d(offset[k]) for k in ("p1", "p2", "o", "t", "b")]
    xa, xp_ = _d(xi)
    out = np.zeros(2)
    F = np.zeros(2)
    det = C.c_double()
    it = C.c_int()
    ok = lib().or_newton_g(*[a[1] for a in arrs], xp_, float(delta), int(max_iter), float(tol_stop), float(tol_succ),
                           out.ctypes.data_as(_dp), C.byref(det), C.byref(it), F.ctypes.data_as(_dp), GAUGES[gauge])
    return bool(ok), out, det.value, it.value, F


def stream_select(w, u):
    wa, wp = _d(w)
    ua, up = _d(u)
    S = C.c_double()
    sel = lib().or_stream_select(wp, up, len(wa), C.byref(S))
    return sel, S.value


def ris_accept(S, w, u):
    """One streaming-resampling step of the pipeline: (accepted, new running sum)."""
    So = C.c_double()
    a = lib().or_ris_accept(float(S), float(w), float(u), C.byref(So))
    return bool(a), So.value


def ris_W(S, phat):
    """The pipeline's unbiased contribution weight of a selected sample: sum of weights / p_hat(y)."""
    return lib().or_ris_W(float(S), float(phat))


def gris_mis(M, T, s, pairwise=False):
    """The pipeline's MIS weight of candidate s in a GRIS merge (confidences M, T_j = p_hat_{<-j}(y_s))."""
    Ma, Mp = _d(M)
    Ta, Tp = _d(T)
    return lib().or_gris_mis(Mp, Tp, len(Ma), int(s), int(bool(pairwise)))


def shift_roundtrip(view: View, params, seed, src, dst):
    out = np.zeros(6)
    pp = params_struct(params)
    rc = lib().or_shift_roundtrip(view.ptr, C.byref(pp), seed, src, dst, out.ctypes.data_as(_dp))
    return rc, out


def shrink_roundtrip(view: View, params, seed, pix, K):
    """Expand pixel `pix`'s stored gated sample K times about the gate centre and shrink it back
    (Sec. 4.4).  Returns (rc, out): out = (J_expand, J_shrink, bary error, tau, tau expanded,
    tau shrunk back, p_hat, p_hat expanded)."""
    out = np.zeros(8)
    pp = params_struct(params)
    rc = lib().or_shrink_roundtrip(view.ptr, C.byref(pp), seed, pix, float(K), out.ctypes.data_as(_dp))
    return rc, out


def ell_sample(geom: Geom, x, q, la, lb, u):
    """One ellipsoidal-connection placement (Sec. 4.4, Sec. 5) from point x toward the light position
    q with l = |x - z| + |z - q| drawn in [la, lb) from the 24 draws u.  Returns None or
    (tri, b1, b2, pdf, z) with pdf the area density of z."""
    out = np.zeros(7)
    (xx, xp), (qq, qp), (uu, up) = _d(x), _d(q), _u(u)
    if not lib().or_ell_sample(geom.ptr, xp, qp, float(la), float(lb), up, out.ctypes.data_as(_dp)):
        return None
    return int(out[0]), out[1], out[2], out[3], out[4:7].copy()


def ell_pdf(geom: Geom, x, q, la, lb, tri, b1, b2):
    """Area density with which the ellipsoidal connection places the point (tri, b1, b2)."""
    (xx, xp), (qq, qp) = _d(x), _d(q)
    return lib().or_ell_pdf(geom.ptr, xp, qp, float(la), float(lb), int(tri), float(b1), float(b2))


def ell_tri_probs(geom: Geom, x, q, ell, nt):
    """Probability of each triangle under the hierarchy walk for the ellipsoid of major axis ell."""
    out = np.zeros(nt)
    (xx, xp), (qq, qp) = _d(x), _d(q)
    lib().or_ell_tri_probs(geom.ptr, xp, qp, float(ell), out.ctypes.data_as(_dp))
    return out
