"""Seeded synthetic scene generators: the inputs of every test, the smoke check and the bench.

This module only builds INPUT DATA (triangle meshes, materials, per-frame rigid transforms,
sensor / emitter poses, gates, reuse parameters).  It holds none of the rendering method's
arithmetic: no ray tracing, no sampling, no path lengths.  Both the CUDA path and the CPU oracle
consume exactly these arrays.

The paper measures on the Bitterli 2016 scenes (Sec. 6), which are not available here; the
generators below stand in for them with the shapes and roles the paper's workloads have:
a closed Lambertian box with an object (Cornell-type interior), a large displaced heightfield
with rigidly moving glossy / diffuse / mirror spheres (dynamic proximity-camera scene), and a
confocal NLOS relay wall with an occluder and a hidden displaced sphere (transient capture).

Conventions
-----------
* Units are metres; optical path length uses c = 1 and refractive index 1 (Sec. 3.1).
* ``materials`` rows are ``(type, albedo, alpha)`` with type 0 = Lambert, 1 = GGX, 2 = mirror.
* ``xforms[f, o]`` is the row-major 3x4 object-to-world matrix of object ``o`` at frame ``f``.
* Sensor ``mode`` 0 = pinhole camera, 1 = confocal scan of a planar wall.
* Emitter ``type`` 0 = isotropic point light, 1 = collimated laser spot, 2 = confocal laser
  (the spot is the scanned wall point of each pixel).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LAMBERT, GGX, MIRROR = 0, 1, 2
PINHOLE, CONFOCAL = 0, 1
EMIT_POINT, EMIT_LASER, EMIT_CONFOCAL = 0, 1, 2

# flags (same bit values on both sides of the library boundary)
FLAG_DIRECT = 1          # include length-1 (direct) candidates
FLAG_NAIVE_SHIFT = 2     # hybrid shift without the path-length Newton correction
FLAG_PAIRWISE_MIS = 4    # pairwise MIS instead of the generalized balance heuristic (2k shifts)
FLAG_GAUGE_AXIS_T = 8    # comparison gauge: fixed axis, the reconnection vertex moves along t
FLAG_GAUGE_AXIS_B = 16   # comparison gauge: fixed axis, the reconnection vertex moves along b
FLAG_GAUGE_START = 32    # comparison gauge: gradient at the start point only (not reversible)
FLAG_TRIANGLE_WALK = 64  # the reconnection vertex may walk across triangle edges during Newton
FLAG_BIN_REUSE = 128     # transient: one pass reusing each pixel's neighbouring bins (Sec. 4.5)
FLAG_ELLIPSOID = 256     # initial candidates also by ellipsoidal path connection, MIS with the path tree


@dataclass
class Params:
    depth: int = 3                 # max number of surface vertices on a path
    n_cand: int = 4                # path trees per pixel
    n_spatial: int = 1             # spatial neighbours per pass
    radius: int = 8                # spatial radius in pixels
    n_spatial_iters: int = 1       # spatial passes
    temporal: int = 0              # temporal reuse on/off
    m_cap: float = 20.0            # confidence cap
    newton_max_iter: int = 5
    newton_tol_frac: float = 0.01  # success threshold, fraction of the gate width
    jac_max: float = 8.0           # shift Jacobian rejection bound
    d_min: float = 0.01            # minimum reconnection segment length (m)
    ray_eps: float = 1e-4          # ray origin offset along the normal (m)
    flags: int = 0
    shrink_k: float = 1.0          # Sec. 4.4 shrink mapping: initial gate widened K times (<= 1: off)
    shrink_fine: int = 0           # trees kept in the gate itself (0: every tree widened, R = 1)


@dataclass
class Scene:
    name: str
    verts: np.ndarray          # float64 [nv, 3] object-local
    tris: np.ndarray           # uint32 [nt, 3]
    tri_object: np.ndarray     # uint32 [nt]
    object_material: np.ndarray  # uint32 [nobj]
    materials: np.ndarray      # float64 [nmat, 3]
    xforms: np.ndarray         # float64 [F, nobj, 12]
    sensors: list              # per frame dict
    emitters: list             # per frame dict
    gates: list                # per frame (L0, dL)  (gated)
    bins: tuple | None         # (t0, width, B)      (transient) or None
    params: Params
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_frames(self) -> int:
        return self.xforms.shape[0]

    @property
    def nt(self) -> int:
        return self.tris.shape[0]

    def frame_xforms(self, f: int) -> np.ndarray:
        return self.xforms[f]

    def crop_sensor(self, f: int):
        return dict(self.sensors[f])


# ----------------------------------------------------------------------------------------------
# mesh primitives
# ----------------------------------------------------------------------------------------------

def _identity34() -> np.ndarray:
    return np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], dtype=np.float64)


def _rot34(axis, angle, pivot) -> np.ndarray:
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    c, s = math.cos(angle), math.sin(angle)
    x, y, z = a
    R = np.array([[c + x * x * (1 - c), x * y * (1 - c) - z * s, x * z * (1 - c) + y * s],
                  [y * x * (1 - c) + z * s, c + y * y * (1 - c), y * z * (1 - c) - x * s],
                  [z * x * (1 - c) - y * s, z * y * (1 - c) + x * s, c + z * z * (1 - c)]])
    p = np.asarray(pivot, dtype=np.float64)
    t = p - R @ p
    return np.concatenate([np.concatenate([R[0], [t[0]]]), np.concatenate([R[1], [t[1]]]),
                           np.concatenate([R[2], [t[2]]])])


def box_mesh(half: float):
    """Closed axis-aligned box [-half, half]^3 as 12 triangles."""
    h = half
    v = np.array([[-h, -h, -h], [h, -h, -h], [h, h, -h], [-h, h, -h],
                  [-h, -h, h], [h, -h, h], [h, h, h], [-h, h, h]], dtype=np.float64)
    f = np.array([[0, 1, 2], [0, 2, 3], [4, 6, 5], [4, 7, 6], [0, 4, 5], [0, 5, 1],
                  [3, 2, 6], [3, 6, 7], [0, 3, 7], [0, 7, 4], [1, 5, 6], [1, 6, 2]], dtype=np.uint32)
    return v, f


def icosphere(subdiv: int):
    """Unit icosphere with 20 * 4**subdiv triangles."""
    t = (1.0 + 5 ** 0.5) / 2.0
    v = [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t],
         [0, 1, -t], [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]]
    v = [list(np.array(p) / np.linalg.norm(p)) for p in v]
    f = [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4],
         [11, 10, 2], [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                p = (np.array(v[a]) + np.array(v[b])) / 2
                v.append(list(p / np.linalg.norm(p)))
                cache[key] = len(v) - 1
            return cache[key]
        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = nf
    return np.array(v, dtype=np.float64), np.array(f, dtype=np.uint32)


def uv_sphere(stacks: int, slices: int):
    """Unit UV sphere: pole fans plus quad rows, 2*slices*(stacks-1) triangles, none degenerate."""
    v = [[0.0, 0.0, 1.0]]
    for i in range(1, stacks):
        th = math.pi * i / stacks
        for j in range(slices):
            ph = 2 * math.pi * j / slices
            v.append([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    v.append([0.0, 0.0, -1.0])
    south = len(v) - 1
    f = []

    def ring(i, j):
        return 1 + (i - 1) * slices + (j % slices)
    for j in range(slices):
        f.append([0, ring(1, j), ring(1, j + 1)])
    for i in range(1, stacks - 1):
        for j in range(slices):
            a, b, c, d = ring(i, j), ring(i + 1, j), ring(i + 1, j + 1), ring(i, j + 1)
            f.append([a, b, c])
            f.append([a, c, d])
    for j in range(slices):
        f.append([south, ring(stacks - 1, j + 1), ring(stacks - 1, j)])
    return np.array(v, dtype=np.float64), np.array(f, dtype=np.uint32)


def _fbm(rng: np.random.Generator, nx: int, ny: int, octaves: int = 5):
    """Seeded fBm on an (nx+1) x (ny+1) lattice from bilinear value noise, range ~[-1, 1]."""
    out = np.zeros((ny + 1, nx + 1))
    amp, total = 1.0, 0.0
    for o in range(octaves):
        cells = 2 ** (o + 2)
        g = rng.uniform(-1, 1, size=(cells + 1, cells + 1))
        ys = np.linspace(0, cells, ny + 1)
        xs = np.linspace(0, cells, nx + 1)
        y0 = np.minimum(ys.astype(int), cells - 1)
        x0 = np.minimum(xs.astype(int), cells - 1)
        fy = (ys - y0)[:, None]
        fx = (xs - x0)[None, :]
        a = g[y0][:, x0]
        b = g[y0][:, x0 + 1]
        c = g[y0 + 1][:, x0]
        d = g[y0 + 1][:, x0 + 1]
        out += amp * ((a * (1 - fx) + b * fx) * (1 - fy) + (c * (1 - fx) + d * fx) * fy)
        total += amp
        amp *= 0.5
    return out / total


def heightfield(rng, nx: int, ny: int, sx: float, sy: float, amp: float):
    """nx x ny cells (2 triangles each) over [-sx/2, sx/2] x [-sy/2, sy/2], z = amp * fBm."""
    h = _fbm(rng, nx, ny)
    h = h / max(1e-9, np.abs(h).max())
    xs = np.linspace(-sx / 2, sx / 2, nx + 1)
    ys = np.linspace(-sy / 2, sy / 2, ny + 1)
    X, Y = np.meshgrid(xs, ys)
    v = np.stack([X.ravel(), Y.ravel(), amp * h.ravel()], axis=1)
    f = []
    for j in range(ny):
        for i in range(nx):
            a = j * (nx + 1) + i
            b, c, d = a + 1, a + nx + 2, a + nx + 1
            f.append([a, b, c])
            f.append([a, c, d])
    return v.astype(np.float64), np.array(f, dtype=np.uint32), h * amp, xs, ys


class _Builder:
    def __init__(self):
        self.v, self.f, self.obj, self.objmat = [], [], [], []
        self.nv = 0

    def add(self, v, f, material):
        oid = len(self.objmat)
        self.v.append(v)
        self.f.append(f + self.nv)
        self.obj.append(np.full(len(f), oid, dtype=np.uint32))
        self.objmat.append(material)
        self.nv += len(v)
        return oid

    def arrays(self):
        return (np.concatenate(self.v).astype(np.float64), np.concatenate(self.f).astype(np.uint32),
                np.concatenate(self.obj).astype(np.uint32), np.array(self.objmat, dtype=np.uint32))


# ----------------------------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------------------------

def box_icosphere(W: int = 64, H: int = 64, seed: int = 0, frames: int = 1) -> Scene:
    """Closed 4 m Lambertian box (albedo 0.7) + 320-triangle icosphere (r = 0.5 m) at a seeded
    position in the inner 2 m cube; coaxial pinhole camera and point light at the origin looking
    down -z, fov 60 deg.  Depth 3, gate L0 = 5.0 m, dL = 0.05 m, 4 path trees, 1 spatial
    neighbour within 8 px, M-cap 20."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    mats = [(LAMBERT, 0.7, 0.0)]
    bv, bf = box_mesh(2.0)
    b.add(bv, bf, 0)
    while True:
        c = rng.uniform(-1.0, 1.0, size=3)
        if np.linalg.norm(c) > 0.9:        # keep the sphere off the camera / light
            break
    alb = rng.uniform(0.3, 0.9)
    mats.append((LAMBERT, alb, 0.0))
    sv, sf = icosphere(2)
    b.add(sv * 0.5 + c, sf, 1)
    v, f, to, om = b.arrays()
    xf = np.tile(_identity34(), (frames, len(om), 1))
    sensor = dict(mode=PINHOLE, pos=[0, 0, 0], fwd=[0, 0, -1], up=[0, 1, 0], fov_y=math.radians(60),
                  W=W, H=H)
    emitter = dict(type=EMIT_POINT, pos=[0, 0, 0], dir=[0, 0, -1], power=10.0)
    p = Params(depth=3, n_cand=4, n_spatial=1, radius=8, n_spatial_iters=1, temporal=0, m_cap=20.0)
    return Scene("box_icosphere", v, f, to, om, np.array(mats, dtype=np.float64), xf,
                 [sensor] * frames, [emitter] * frames, [(5.0, 0.05)] * frames, None, p, seed,
                 meta=dict(sphere_centre=c.tolist()))


def heightfield_spheres(W: int = 512, H: int = 512, frames: int = 32, seed: int = 1,
                        nx: int = 200, ny: int = 125, n_spheres: int = 20,
                        sphere_stacks: int = 21, sphere_slices: int = 20,
                        extent=(20.0, 12.5), cam=(0.0, -3.6, 1.7), look=(0.0, 0.8, 0.2)) -> Scene:
    """Dynamic time-gated workload: a 200 x 125-cell fBm heightfield (50,000 triangles, 20 m x
    12.5 m, amplitude 0.2 m) plus 20 spheres of 800 triangles (radius U[0.4, 0.95] m) resting on it
    within a few metres of the sensor, each rotating rigidly 1 deg/frame about a seeded axis through a
    seeded pivot within 2 m.  Materials per object: GGX (alpha ~ U[0.05, 0.5]) on 70 %, Lambert on
    20 %, mirror on 10 %; the heightfield is one of the Lambertian objects.  A coaxial camera and
    point light 1.7 m above the ground look into the cluster (a proximity time-gated sensor).
    Depth 4, temporal + 5 spatial neighbours within 30 px, M-cap 20, L0 = 8 m, dL = 0.03 m."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    sx, sy = extent
    hv, hf, hgrid, xs, ys = heightfield(rng, nx, ny, sx, sy, 0.2)
    nobj = 1 + n_spheres
    n_ggx = int(round(0.7 * nobj))
    n_mir = max(1, int(round(0.1 * nobj)))
    n_lam = nobj - n_ggx - n_mir
    kinds = [LAMBERT] * (n_lam - 1) + [GGX] * n_ggx + [MIRROR] * n_mir
    rng.shuffle(kinds)
    kinds = [LAMBERT] + kinds            # object 0 (heightfield) is Lambertian
    mats = []
    for k in kinds:
        alb = rng.uniform(0.3, 0.9)
        alpha = rng.uniform(0.05, 0.5) if k == GGX else 0.0
        mats.append((k, alb, alpha))
    b.add(hv, hf, 0)
    sv, sf = uv_sphere(sphere_stacks, sphere_slices)
    centres, axes, pivots = [], [], []
    for s in range(n_spheres):
        rad = rng.uniform(0.4, 0.95)
        cx = rng.uniform(-2.2, 2.2)
        cy = rng.uniform(-0.6, 2.2)
        i = int(np.clip(round((cx + sx / 2) / sx * nx), 0, nx))
        j = int(np.clip(round((cy + sy / 2) / sy * ny), 0, ny))
        c = np.array([cx, cy, hgrid[j, i] + rad])
        centres.append(c)
        b.add(sv * rad + c, sf, 1 + s)
        ax = rng.normal(size=3)
        axes.append(ax / np.linalg.norm(ax))
        off = rng.normal(size=3)
        off[2] = 0.0
        off = off / max(1e-9, np.linalg.norm(off)) * rng.uniform(0.0, 2.0)
        pivots.append(c + off)
    v, f, to, om = b.arrays()
    xf = np.zeros((frames, nobj, 12))
    for fr in range(frames):
        xf[fr, 0] = _identity34()
        for s in range(n_spheres):
            ang = math.radians(1.0) * fr
            # even spheres orbit a nearly vertical axis through their pivot (staying near the
            # ground), odd spheres spin about a seeded axis through their centre
            xf[fr, 1 + s] = _rot34([0.15 * axes[s][0], 0.15 * axes[s][1], 1.0], ang, pivots[s]) \
                if s % 2 == 0 else _rot34(axes[s], ang, centres[s])
    fwd = np.array(look, dtype=float) - np.array(cam, dtype=float)
    fwd /= np.linalg.norm(fwd)
    sensor = dict(mode=PINHOLE, pos=list(cam), fwd=list(fwd), up=[0, 0, 1], fov_y=math.radians(60), W=W, H=H)
    emitter = dict(type=EMIT_POINT, pos=list(cam), dir=list(fwd), power=20.0)
    p = Params(depth=4, n_cand=4, n_spatial=5, radius=30, n_spatial_iters=1, temporal=1, m_cap=20.0)
    return Scene("heightfield_spheres", v, f, to, om, np.array(mats, dtype=np.float64), xf,
                 [sensor] * frames, [emitter] * frames, [(8.0, 0.03)] * frames, None, p, seed,
                 meta=dict(centres=np.array(centres).tolist(), kinds=kinds))


def confocal_nlos(W: int = 256, H: int = 256, frames: int = 16, seed: int = 2, B: int = 1024,
                  stacks: int = 224, slices: int = 224) -> Scene:
    """Transient confocal NLOS workload: 2 m x 2 m Lambertian relay wall (z = 0, albedo 0.8,
    tessellated 16 x 16), a 1.5 m square occluder (plane x = 1, albedo 0.5) that hides a seeded
    ~100k-triangle displaced sphere (r = 0.3 m +- 0.05 m, albedo 0.7, centre 1 m in front of the
    wall) from the device at (2, 0, 1).  Confocal 256 x 256 scan of the wall, 1024 bins of 1 mm
    measuring L - 2 |device - wall point| from t0 = 1.35 m, depth 4, 8 path trees, temporal + 3
    spatial neighbours within 10 px; the device translates 5 mm/frame along +y."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    mats = [(LAMBERT, 0.8, 0.0), (LAMBERT, 0.5, 0.0), (LAMBERT, 0.7, 0.0)]
    n = 16
    xs = np.linspace(-1, 1, n + 1)
    X, Y = np.meshgrid(xs, xs)
    wv = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    wf = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            wf += [[a, a + 1, a + n + 2], [a, a + n + 2, a + n + 1]]
    b.add(wv, np.array(wf, dtype=np.uint32), 0)
    ov = np.array([[1.0, -0.75, 0.7], [1.0, 0.75, 0.7], [1.0, 0.75, 2.2], [1.0, -0.75, 2.2]])
    b.add(ov, np.array([[0, 1, 2], [0, 2, 3]], dtype=np.uint32), 1)
    sv, sf = uv_sphere(stacks, slices)
    k = rng.normal(size=(6, 3))
    ph = rng.uniform(0, 2 * math.pi, size=6)
    disp = np.zeros(len(sv))
    for i in range(6):
        disp += np.sin(3.0 * (sv @ k[i]) + ph[i])
    disp = 0.05 * disp / max(1e-9, np.abs(disp).max())
    sv = sv * (0.3 + disp)[:, None] + np.array([0.0, 0.0, 1.0])
    b.add(sv, sf, 2)
    v, f, to, om = b.arrays()
    xf = np.tile(_identity34(), (frames, len(om), 1))
    sensors = []
    for fr in range(frames):
        sensors.append(dict(mode=CONFOCAL, pos=[2.0, 0.005 * fr, 1.0], fwd=[-1, 0, 0], up=[0, 0, 1],
                            fov_y=0.0, W=W, H=H, wall_o=[-1.0, -1.0, 0.0], wall_u=[2.0, 0.0, 0.0],
                            wall_v=[0.0, 2.0, 0.0]))
    emitters = [dict(type=EMIT_CONFOCAL, pos=s["pos"], dir=[-1, 0, 0], power=1.0) for s in sensors]
    p = Params(depth=4, n_cand=8, n_spatial=3, radius=10, n_spatial_iters=1, temporal=1, m_cap=20.0)
    return Scene("confocal_nlos", v, f, to, om, np.array(mats, dtype=np.float64), xf, sensors,
                 emitters, [(1.35, 0.001)] * frames, (1.35, 0.001, B), p, seed)


def box_materials(W: int = 32, H: int = 32, seed: int = 0, frames: int = 1, sphere_alpha: float = 0.1,
                  moving: bool = False) -> Scene:
    """The 4 m box with one material per wall (floor mirror, back wall GGX alpha 0.3, ceiling
    GGX alpha 0.12, other walls Lambert) and a GGX icosphere of roughness ``sphere_alpha``;
    exercises random replay through glossy and specular vertices.  With ``moving`` the sphere
    rotates 2 deg/frame about an axis through a point 0.6 m from its centre."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    mats = [(LAMBERT, 0.7, 0.0), (MIRROR, 0.8, 0.0), (GGX, 0.8, 0.3), (GGX, 0.7, 0.12), (LAMBERT, 0.5, 0.0),
            (GGX, 0.75, sphere_alpha)]
    bv, bf = box_mesh(2.0)
    wall_mat = [0, 1, 2, 3, 4, 0]          # -z (back), +z... per pair of triangles
    for w in range(6):
        b.add(bv, bf[2 * w:2 * w + 2], wall_mat[w])
    c = np.array([0.4, -0.8, -1.2])
    sv, sf = icosphere(2)
    b.add(sv * 0.5 + c, sf, 5)
    v, f, to, om = b.arrays()
    nobj = len(om)
    xf = np.tile(_identity34(), (frames, nobj, 1))
    if moving:
        for fr in range(frames):
            xf[fr, nobj - 1] = _rot34([0.3, 1.0, 0.2], math.radians(2.0) * fr, c + np.array([0.6, 0.0, 0.0]))
    sensor = dict(mode=PINHOLE, pos=[0, 0, 0], fwd=[0, 0, -1], up=[0, 1, 0], fov_y=math.radians(60), W=W, H=H)
    emitter = dict(type=EMIT_POINT, pos=[0, 0, 0], dir=[0, 0, -1], power=10.0)
    p = Params(depth=4, n_cand=4, n_spatial=2, radius=4, n_spatial_iters=1, temporal=0, m_cap=20.0)
    return Scene("box_materials", v, f, to, om, np.array(mats, dtype=np.float64), xf, [sensor] * frames,
                 [emitter] * frames, [(6.5, 0.5)] * frames, None, p, seed)


def white_furnace_sphere(R: float = 1.0, albedo: float = 0.5, subdiv: int = 5, W: int = 16,
                         H: int = 16) -> Scene:
    """Closed Lambertian icosphere of radius R with a coaxial camera and point light at its
    centre (a closed-form check of the path-integral estimator)."""
    sv, sf = icosphere(subdiv)
    b = _Builder()
    b.add(sv * R, sf, 0)
    v, f, to, om = b.arrays()
    xf = np.tile(_identity34(), (1, 1, 1))
    sensor = dict(mode=PINHOLE, pos=[0, 0, 0], fwd=[0, 0, -1], up=[0, 1, 0], fov_y=math.radians(40),
                  W=W, H=H)
    emitter = dict(type=EMIT_POINT, pos=[0, 0, 0], dir=[0, 0, -1], power=1.0)
    p = Params(depth=3, n_cand=1, n_spatial=0, temporal=0)
    return Scene("white_furnace", v, f, to, om, np.array([(LAMBERT, albedo, 0.0)]), xf, [sensor],
                 [emitter], [(0.0, 1e9)], None, p, 0)


def lambert_plane(W: int = 8, H: int = 8, albedo: float = 0.6, z: float = -2.0,
                  light=(0.3, 0.0, 0.0)) -> Scene:
    """One large Lambertian plane z = const facing a pinhole camera at the origin, with a point
    light at ``light`` (single-bounce closed form)."""
    s = 100.0
    v = np.array([[-s, -s, z], [s, -s, z], [s, s, z], [-s, s, z]], dtype=np.float64)
    f = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.uint32)
    xf = np.tile(_identity34(), (1, 1, 1))
    sensor = dict(mode=PINHOLE, pos=[0, 0, 0], fwd=[0, 0, -1], up=[0, 1, 0], fov_y=math.radians(30),
                  W=W, H=H)
    emitter = dict(type=EMIT_POINT, pos=list(light), dir=[0, 0, -1], power=1.0)
    p = Params(depth=1, n_cand=1, n_spatial=0, temporal=0, flags=FLAG_DIRECT)
    return Scene("lambert_plane", v, f, np.zeros(2, dtype=np.uint32), np.zeros(1, dtype=np.uint32),
                 np.array([(LAMBERT, albedo, 0.0)]), xf, [sensor], [emitter], [(4.0, 0.05)], None,
                 p, 0)


def batch_instances(n: int = 64, seed: int = 3, max_res: int = 1024, min_res: int = 64):
    """Batched workload description: per instance (scene index, W, H, dL, depth), resolutions
    log-uniform in [64, 1024], gate widths U[0.01, 0.1] m, depths U{2..5}, 4 scene variants."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        res = int(round(math.exp(rng.uniform(math.log(min_res), math.log(max_res)))))
        out.append(dict(scene=int(rng.integers(0, 4)), W=res, H=res, dL=float(rng.uniform(0.01, 0.1)),
                        depth=int(rng.integers(2, 6)), seed=int(rng.integers(0, 2 ** 31))))
    return out
