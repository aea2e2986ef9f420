"""Procedural box-room scenes, camera shading points and one-bounce VPLs.

Geometry: the room is the unit cube [0,1]^3 with y up.  Five walls are present
(floor y=0, ceiling y=1, x=0, x=1, back z=1); the front z=0 is open and the
camera looks through it.  Occluders are axis-aligned boxes strictly inside the
room.  Every face carries a scalar albedo drawn from U[0.2, 0.8] and, on a
``glossy_frac`` share of faces, a Phong exponent drawn from U[10, 100]
(exponent 0 means diffuse).

A 0.2 x 0.2 area light sits at the centre of the ceiling and emits downwards.
VPLs are the first surface hits of cosine-distributed rays leaving uniform points
on the light (instant radiosity, one bounce); each keeps the position, the normal
of the face it landed on, that face's albedo and exponent, the direction back
towards the light, and the flux power/N_emitted.

Shading points are the first hits of one ray per pixel from a pinhole camera at
(0.5, 0.5, -1.35) looking +z with a 40 degree vertical field of view.

Array layouts (float32, "three float4 planes"):
  points[3, m, 4]: [px py pz albedo] [nx ny nz gloss] [ox oy oz 0]   (o = unit dir to camera)
  vpls  [3, n, 4]: [px py pz albedo] [nx ny nz gloss] [ix iy iz flux] (i = unit dir to light)
  boxes [nb, 6]  : [xmin ymin zmin xmax ymax zmax]

Colour (cfg["rgb"] true): every face also draws an RGB albedo from U[0.2, 0.8]^3 (a
separate seeded stream, so the geometry and the VPLs stay those of the grey scene)
and the light has colour cfg["light_rgb"]; the scalar albedo and flux then become
the Rec. 709 luminances of the colours, and ``Scene.rgb`` holds point_albedo [m, 3],
vpl_albedo [n, 3] and vpl_flux [n, 3] (float32).

Meshes (cfg["n_meshes"] > 0): that many icospheres (the icosahedron subdivided
cfg["mesh_subdiv"] times, vertices pushed to the sphere) stand on the floor as
triangle occluders; each sphere is one material (face id after the boxes' faces),
shading points and VPLs on it take the flat normal of the triangle they hit, facing
the incoming ray.  ``Scene.tris`` holds them as [nt, 3, 3] float32.

Everything here is input generation: the nearest-hit ray caster below only places
points and lights.  It uses numpy's PCG64 generator seeded per scene.
"""
from __future__ import annotations

import dataclasses
import math

import os

import numpy as np

CAMERA_POS = np.array([0.5, 0.5, -1.35])
LUMINANCE = np.array([0.2126, 0.7152, 0.0722])  # Rec. 709 weights of R, G, B
CAMERA_VFOV_DEG = 40.0

# wall ids 0..4: floor, ceiling, x=0, x=1, back
_WALL_NORMALS = np.array([[0, 1, 0], [0, -1, 0], [1, 0, 0], [-1, 0, 0], [0, 0, -1]], dtype=np.float64)


@dataclasses.dataclass
class Scene:
    cfg: dict
    boxes: np.ndarray          # [nb, 6] float32
    points: np.ndarray         # [3, m, 4] float32
    vpls: np.ndarray           # [3, n, 4] float32
    width: int
    height: int
    n_emitted: int
    rgb: dict | None = None    # colour arrays of an RGB scene (see the module notes)
    tris: np.ndarray | None = None  # [nt, 3, 3] triangle occluders of a mesh scene

    @property
    def occluders(self):
        """What shadow rays test: the boxes, or (boxes, triangles) in a mesh scene."""
        return self.boxes if self.tris is None else (self.boxes, self.tris)

    @property
    def m(self) -> int:
        return self.points.shape[1]

    @property
    def n(self) -> int:
        return self.vpls.shape[1]

    @property
    def nb(self) -> int:
        return self.boxes.shape[0]


def _make_boxes(cfg: dict, rng: np.random.Generator) -> np.ndarray:
    boxes = []
    nbig = int(cfg.get("n_big_boxes", 0))
    for k in range(nbig):
        # large boxes standing on the floor, one per horizontal band of x
        sx, sz = rng.uniform(0.18, 0.32, size=2)
        sy = rng.uniform(0.25, 0.6)
        band = (k + 0.5) / nbig
        cx = np.clip(band + rng.uniform(-0.08, 0.08), sx / 2 + 0.05, 1 - sx / 2 - 0.05)
        cz = rng.uniform(0.35 + sz / 2, 0.9 - sz / 2)
        boxes.append([cx - sx / 2, 0.0, cz - sz / 2, cx + sx / 2, sy, cz + sz / 2])
    for _ in range(int(cfg.get("n_small_boxes", 0))):
        s = rng.uniform(0.02, 0.15, size=3)
        lo = rng.uniform(0.01, 1.0 - 0.01 - s)
        lo[1] = rng.uniform(0.01, 0.9 - s[1])  # keep the light and the ceiling clear
        boxes.append([lo[0], lo[1], lo[2], lo[0] + s[0], lo[1] + s[1], lo[2] + s[2]])
    if not boxes:
        return np.zeros((0, 6), dtype=np.float32)
    return np.asarray(boxes, dtype=np.float32)


_ICO_T = (1.0 + 5.0 ** 0.5) / 2.0
_ICO_V = [(-1, _ICO_T, 0), (1, _ICO_T, 0), (-1, -_ICO_T, 0), (1, -_ICO_T, 0), (0, -1, _ICO_T), (0, 1, _ICO_T),
          (0, -1, -_ICO_T), (0, 1, -_ICO_T), (_ICO_T, 0, -1), (_ICO_T, 0, 1), (-_ICO_T, 0, -1), (-_ICO_T, 0, 1)]
_ICO_F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6),
          (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
          (8, 6, 7), (9, 8, 1)]


def icosphere(subdiv: int) -> np.ndarray:
    """Triangles [nt, 3, 3] of the unit icosphere: each subdivision splits a triangle
    into four at its edge midpoints, pushed out to the sphere."""
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in _ICO_V]
    faces = list(_ICO_F)
    for _ in range(subdiv):
        mid = {}

        def m(i, j):
            key = (min(i, j), max(i, j))
            if key not in mid:
                v = verts[i] + verts[j]
                verts.append(v / np.linalg.norm(v))
                mid[key] = len(verts) - 1
            return mid[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = m(a, b), m(b, c), m(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    return V[np.array(faces)]


def _make_meshes(cfg: dict, rng: np.random.Generator, boxes: np.ndarray):
    """(triangles [nt, 3, 3] float32, bounding spheres [(centre, radius)]) or (None, [])."""
    n = int(cfg.get("n_meshes", 0))
    if n <= 0:
        return None, []
    unit = icosphere(int(cfg.get("mesh_subdiv", 2)))
    out, spheres = [], []
    for k in range(n):
        r = rng.uniform(0.07, 0.14)
        cx = (k + 0.5) / n + rng.uniform(-0.05, 0.05)
        cx = float(np.clip(cx, r + 0.02, 1 - r - 0.02))
        cz = rng.uniform(0.3 + r, 0.9 - r)
        cy = r + rng.uniform(0.0, 0.25)
        centre = np.array([cx, cy, cz])
        out.append(unit * r + centre)
        spheres.append((centre, r))
    return np.concatenate(out).astype(np.float32), spheres


def _tri_nearest(org, d, tris, spheres, chunk=1024):
    """Nearest hit of rays with the triangles (float64 Moller-Trumbore): (t, index).
    Each mesh is tested only against the rays that meet its bounding sphere."""
    nr = org.shape[0]
    t_out = np.full(nr, np.inf)
    i_out = np.full(nr, -1, dtype=np.int64)
    T = tris.astype(np.float64)
    per = T.shape[0] // max(len(spheres), 1)
    for m, (c, r) in enumerate(spheres):
        # rays through the (slightly inflated) bounding sphere
        oc = org - c
        b = np.sum(oc * d, axis=1)
        cc = np.sum(oc * oc, axis=1) - (1.001 * r) ** 2
        dd2 = np.sum(d * d, axis=1)
        disc = b * b - dd2 * cc
        rays = np.nonzero(disc >= 0)[0]
        if rays.size == 0:
            continue
        Tm = T[m * per:(m + 1) * per]
        v0, e1, e2 = Tm[:, 0], Tm[:, 1] - Tm[:, 0], Tm[:, 2] - Tm[:, 0]
        for s in range(0, rays.size, chunk):
            idx = rays[s:s + chunk]
            D = d[idx, None, :]
            p = np.cross(D, e2[None])
            det = np.sum(e1[None] * p, axis=-1)
            with np.errstate(divide="ignore", invalid="ignore"):
                inv = 1.0 / det
                sv = org[idx, None, :] - v0[None]
                u = np.sum(sv * p, axis=-1) * inv
                q = np.cross(sv, e1[None])
                v = np.sum(D * q, axis=-1) * inv
                t = np.sum(e2[None] * q, axis=-1) * inv
            ok = (det != 0) & (u >= 0) & (u <= 1) & (v >= 0) & (u + v <= 1) & (t > 1e-7)
            t = np.where(ok, t, np.inf)
            j = np.argmin(t, axis=1)
            tj = t[np.arange(idx.size), j]
            better = tj < t_out[idx]
            t_out[idx] = np.where(better, tj, t_out[idx])
            i_out[idx] = np.where(better, m * per + j, i_out[idx])
    return t_out, i_out


def _materials(n_faces: int, glossy_frac: float, rng: np.random.Generator):
    albedo = rng.uniform(0.2, 0.8, size=n_faces)
    gloss = np.zeros(n_faces)
    if glossy_frac > 0:
        sel = rng.uniform(size=n_faces) < glossy_frac
        gloss[sel] = rng.uniform(10.0, 100.0, size=int(sel.sum()))
    return albedo, gloss


# Ray-box work above which the nearest-hit search is split over host processes (the
# rays are independent, so the result is the same bits as one process gives).
_POOL_WORK = 50_000_000


def _nearest_hit_part(args):
    return _nearest_hit_serial(*args)


def _nearest_hit(org: np.ndarray, d: np.ndarray, boxes: np.ndarray, chunk: int = 2048, procs: int | None = None):
    """Nearest surface hit of rays (org, d) in the room (float64).

    Returns (t, face) where face in [0,5) is a wall, 5 + 6*b + f is face f
    (-x,+x,-y,+y,-z,+z) of box b, and -1 means the ray left through the opening.
    Large searches run on ``procs`` spawned processes (default: the host cores, at
    most 16), each on a contiguous share of the rays.
    """
    nr = org.shape[0]
    if procs is None:
        procs = min(16, os.cpu_count() or 1) if nr * max(boxes.shape[0], 1) >= _POOL_WORK else 1
    if procs > 1 and nr >= 2 * chunk:
        import multiprocessing
        cuts = np.linspace(0, nr, procs + 1).astype(np.int64)
        parts = [(org[a:b], d[a:b], boxes, chunk) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
        with multiprocessing.get_context("spawn").Pool(len(parts)) as pool:
            res = pool.map(_nearest_hit_part, parts)
        return np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res])
    return _nearest_hit_serial(org, d, boxes, chunk)


def _nearest_hit_serial(org: np.ndarray, d: np.ndarray, boxes: np.ndarray, chunk: int = 2048):
    nr = org.shape[0]
    t_out = np.full(nr, np.inf)
    face_out = np.full(nr, -1, dtype=np.int64)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        # exit of the room cube
        t0 = (0.0 - org) * inv
        t1 = (1.0 - org) * inv
        tfar = np.where(d > 0, t1, np.where(d < 0, t0, np.inf))
        axis = np.argmin(tfar, axis=1)
        texit = tfar[np.arange(nr), axis]
        sign = d[np.arange(nr), axis] > 0
        # walls: floor(y-)=0, ceiling(y+)=1, x-=2, x+=3, back(z+)=4, front(z-)=open
        wall = np.select(
            [(axis == 1) & ~sign, (axis == 1) & sign, (axis == 0) & ~sign,
             (axis == 0) & sign, (axis == 2) & sign],
            [0, 1, 2, 3, 4], default=-1)
        t_out[:] = texit
        face_out[:] = wall
        if boxes.shape[0]:
            bl = boxes[:, :3].astype(np.float64)
            bh = boxes[:, 3:].astype(np.float64)
            for s in range(0, nr, chunk):
                e = min(nr, s + chunk)
                o = org[s:e, None, :]
                iv = inv[s:e, None, :]
                ta = (bl[None] - o) * iv
                tb = (bh[None] - o) * iv
                tn = np.minimum(ta, tb)
                tf = np.maximum(ta, tb)
                tn = np.where(np.isnan(tn), -np.inf, tn)
                tf = np.where(np.isnan(tf), np.inf, tf)
                tnear = tn.max(axis=2)
                tfar_b = tf.min(axis=2)
                hit = (tnear <= tfar_b) & (tnear > 1e-7)
                tn_h = np.where(hit, tnear, np.inf)
                bidx = np.argmin(tn_h, axis=1)
                tb_min = tn_h[np.arange(e - s), bidx]
                better = tb_min < t_out[s:e]
                ax = np.argmax(tn[np.arange(e - s), bidx], axis=1)
                dsign = d[s:e][np.arange(e - s), ax] > 0
                # entering through the face whose normal opposes the ray
                f = 2 * ax + np.where(dsign, 0, 1)
                t_out[s:e] = np.where(better, tb_min, t_out[s:e])
                face_out[s:e] = np.where(better, 5 + 6 * bidx + f, face_out[s:e])
    return t_out, face_out


def _face_normals(face: np.ndarray) -> np.ndarray:
    nrm = np.zeros((face.shape[0], 3))
    w = face < 5
    nrm[w] = _WALL_NORMALS[face[w]]
    b = ~w
    f = (face[b] - 5) % 6
    ax = f // 2
    sgn = np.where(f % 2 == 0, -1.0, 1.0)
    nb = np.zeros((f.shape[0], 3))
    nb[np.arange(f.shape[0]), ax] = sgn
    nrm[b] = nb
    return nrm


def _camera_rays(width: int, height: int):
    tan_half = math.tan(math.radians(CAMERA_VFOV_DEG) / 2)
    aspect = width / height
    py, px = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    u = ((px + 0.5) / width * 2 - 1) * tan_half * aspect
    v = (1 - (py + 0.5) / height * 2) * tan_half
    d = np.stack([u, v, np.ones_like(u)], axis=-1).reshape(-1, 3)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    org = np.broadcast_to(CAMERA_POS, d.shape).copy()
    return org, d


def make_scene(cfg: dict, seed: int | None = None) -> Scene:
    """Build the scene, shading points and VPLs of preset ``cfg`` (deterministic in ``seed``)."""
    seed = int(cfg["scene_seed"] if seed is None else seed)
    rng = np.random.default_rng(seed)
    boxes = _make_boxes(cfg, rng)
    nb = boxes.shape[0]
    albedo, gloss = _materials(5 + 6 * nb, float(cfg.get("glossy_frac", 0.0)), rng)
    # meshes draw from their own stream, so the scenes without them are unchanged
    mrng = np.random.default_rng(seed + 104729)
    tris, spheres = _make_meshes(cfg, mrng, boxes)
    n_mesh = int(cfg.get("n_meshes", 0)) if tris is not None else 0
    per_mesh = tris.shape[0] // max(n_mesh, 1) if tris is not None else 0
    if n_mesh:
        ma, mg = _materials(n_mesh, float(cfg.get("glossy_frac", 0.0)), mrng)
        albedo, gloss = np.concatenate([albedo, ma]), np.concatenate([gloss, mg])
    colour = bool(cfg.get("rgb", False))
    if colour:
        face_rgb = np.random.default_rng(seed + 7919).uniform(0.2, 0.8, size=(5 + 6 * nb, 3))
        if n_mesh:
            face_rgb = np.concatenate([face_rgb, mrng.uniform(0.2, 0.8, size=(n_mesh, 3))])
        albedo = face_rgb @ LUMINANCE
        light_rgb = np.asarray(cfg.get("light_rgb", (1.0, 0.85, 0.7)), dtype=np.float64)

    def hit(o, dd):
        """Nearest hit over walls, boxes and triangles: (t, face, normal)."""
        t, face = _nearest_hit(o, dd, boxes)
        nrm = np.zeros((t.shape[0], 3))
        if tris is not None:
            tt, ti = _tri_nearest(o, dd, tris, spheres)
            closer = tt < t
            t = np.where(closer, tt, t)
            face = np.where(closer, 5 + 6 * nb + ti // per_mesh, face)
            T = tris[ti[closer]].astype(np.float64)
            n = np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0])
            n /= np.linalg.norm(n, axis=1, keepdims=True)
            n = np.where(np.sum(n * dd[closer], axis=1, keepdims=True) > 0, -n, n)
            nrm[closer] = n
        flat = face < 5 + 6 * nb
        nrm[flat & (face >= 0)] = _face_normals(face[flat & (face >= 0)])
        return t, face, nrm

    # shading points
    width, height = int(cfg["width"]), int(cfg["height"])
    org, d = _camera_rays(width, height)
    t, face, nrm = hit(org, d)
    if np.any(face < 0):
        raise RuntimeError("a camera ray missed the room")
    pos = org + t[:, None] * d
    m = pos.shape[0]
    points = np.zeros((3, m, 4), dtype=np.float32)
    points[0, :, :3] = pos
    points[0, :, 3] = albedo[face]
    points[1, :, :3] = nrm
    points[1, :, 3] = gloss[face]
    points[2, :, :3] = -d

    # VPLs: one bounce from the ceiling light, flux = power / rays emitted
    n = int(cfg["n_vpl"])
    half = float(cfg.get("light_size", 0.2)) / 2
    power = float(cfg.get("light_power", 1.0))
    hits_pos, hits_face, hits_dir, hits_nrm = [], [], [], []
    n_hit = 0
    n_emitted = 0
    batch = max(1024, n)
    while n_hit < n:
        r = rng.uniform(size=(batch, 4))
        lo = np.stack([0.5 - half + 2 * half * r[:, 0], np.ones(batch), 0.5 - half + 2 * half * r[:, 1]], axis=1)
        phi = 2 * math.pi * r[:, 2]
        sin_t = np.sqrt(r[:, 3])
        cos_t = np.sqrt(1 - r[:, 3])
        dd = np.stack([sin_t * np.cos(phi), -cos_t, sin_t * np.sin(phi)], axis=1)
        tt, ff, nn = hit(lo, dd)
        ok = ff >= 0
        # keep emission order so that N_emitted is well defined
        idx = np.nonzero(ok)[0]
        need = n - n_hit
        if idx.shape[0] >= need:
            last = idx[need - 1]
            idx = idx[:need]
            n_emitted += last + 1
        else:
            n_emitted += batch
        hits_pos.append(lo[idx] + tt[idx, None] * dd[idx])
        hits_face.append(ff[idx])
        hits_dir.append(-dd[idx])
        hits_nrm.append(nn[idx])
        n_hit += idx.shape[0]
    vpos = np.concatenate(hits_pos)[:n]
    vface = np.concatenate(hits_face)[:n]
    vdir = np.concatenate(hits_dir)[:n]
    vnrm = np.concatenate(hits_nrm)[:n]
    vpls = np.zeros((3, n, 4), dtype=np.float32)
    vpls[0, :, :3] = vpos
    vpls[0, :, 3] = albedo[vface]
    vpls[1, :, :3] = vnrm
    vpls[1, :, 3] = gloss[vface]
    vpls[2, :, :3] = vdir
    vpls[2, :, 3] = power / n_emitted
    rgb = None
    if colour:
        vpls[2, :, 3] = power / n_emitted * float(light_rgb @ LUMINANCE)
        rgb = dict(point_albedo=face_rgb[face].astype(np.float32),
                   vpl_albedo=face_rgb[vface].astype(np.float32),
                   vpl_flux=np.broadcast_to(power / n_emitted * light_rgb, (n, 3)).astype(np.float32))
    return Scene(cfg=cfg, boxes=boxes, points=points, vpls=vpls, width=width, height=height,
                 n_emitted=int(n_emitted), rgb=rgb, tris=tris)


def single_quad_scene(vpl_pos, vpl_nrm, vpl_flux, vpl_albedo, quad_y: float, res: int,
                      quad_albedo: float, extent: float = 1.0):
    """One VPL above one horizontal quad, no occluders (closed-form test input).

    Shading points are the centres of a ``res`` x ``res`` grid over the quad
    [0,extent]^2 at height ``quad_y`` with normal +y, viewed from straight above.
    """
    xs = (np.arange(res) + 0.5) / res * extent
    gx, gz = np.meshgrid(xs, xs, indexing="ij")
    m = res * res
    points = np.zeros((3, m, 4), dtype=np.float32)
    points[0, :, 0] = gx.ravel()
    points[0, :, 1] = quad_y
    points[0, :, 2] = gz.ravel()
    points[0, :, 3] = quad_albedo
    points[1, :, 1] = 1.0
    points[2, :, 1] = 1.0
    vpls = np.zeros((3, 1, 4), dtype=np.float32)
    vpls[0, 0, :3] = vpl_pos
    vpls[0, 0, 3] = vpl_albedo
    vpls[1, 0, :3] = vpl_nrm
    vpls[2, 0, :3] = vpl_nrm
    vpls[2, 0, 3] = vpl_flux
    return points, vpls


_CACHE_FIELDS = ("boxes", "points", "vpls")


def load_or_make_scene(cfg: dict, cache_dir: str | None = None) -> Scene:
    """make_scene(cfg), stored in and reloaded from ``cache_dir`` (an .npz per scene
    recipe) so that large scenes are generated once; None: no cache."""
    if cache_dir is None or cfg.get("rgb") or int(cfg.get("n_meshes", 0)):
        return make_scene(cfg)
    import hashlib
    import json
    import os
    keys = ("width", "height", "n_vpl", "n_big_boxes", "n_small_boxes", "glossy_frac", "scene_seed",
            "light_power", "light_size")
    tag = hashlib.sha1(json.dumps({k: cfg.get(k) for k in keys}, sort_keys=True).encode()).hexdigest()[:16]
    path = os.path.join(cache_dir, f"scene_{tag}.npz")
    if os.path.exists(path):
        z = np.load(path)
        return Scene(cfg=cfg, boxes=z["boxes"], points=z["points"], vpls=z["vpls"], width=int(cfg["width"]),
                     height=int(cfg["height"]), n_emitted=int(z["n_emitted"]))
    sc = make_scene(cfg)
    os.makedirs(cache_dir, exist_ok=True)
    np.savez(path + ".tmp.npz", boxes=sc.boxes, points=sc.points, vpls=sc.vpls, n_emitted=sc.n_emitted)
    os.replace(path + ".tmp.npz", path)
    return sc
