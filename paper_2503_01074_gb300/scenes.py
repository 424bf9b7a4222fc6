"""Seeded synthetic scene, sensor and trajectory generators.

This module produces *inputs* only: FP32 vertex arrays, int32 triangle and
material arrays, material reflectivity tables and sensor poses.  It holds
none of the sonar method's arithmetic (no ray casting, scoring, binning,
noise, normalisation or resampling), so both the CUDA path and the FP64
oracle can be fed from it without sharing any of the method's code.

The scenes stand in for the paper's photogrammetry and Sketchfab scenes
(towing tank, pier, mall; Sec. III-C), which are not available: a seabed
heightfield (fractional Brownian motion over value noise), pier piles
(16-sided cylinders), boxes, an icosphere and a flat quad.  Sensor defaults
follow the Oculus M750-d field of view the paper uses (130 deg x 20 deg,
Sec. III-A-2).

World frame: z up; a sensor with zero yaw looks along +y; x is to its right.
A pose is a sensor->world rotation R (row-major 3x3) and a position.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh", "SensorSpec", "quad", "icosphere", "heightfield", "cylinder", "box",
    "merge", "pose_matrix", "tiny_scene", "single_frame_scene", "random_soup",
    "sensor_tiny", "sensor_single", "trajectory", "batched_workload",
    "large_scene", "materials_uniform", "height_function",
]


@dataclass
class Mesh:
    """A triangle soup: verts [V,3] f32, tris [T,3] i32 (counter-clockwise
    seen from outside), mat [T] i32 material ids."""
    verts: np.ndarray
    tris: np.ndarray
    mat: np.ndarray
    info: dict = field(default_factory=dict)

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


@dataclass
class SensorSpec:
    """Sonar geometry and pose, mirroring the C-ABI `sonar_sensor` struct."""
    pos: np.ndarray            # [3] f32
    rot: np.ndarray            # [3,3] f32, sensor->world
    n_beams: int
    n_elev: int
    n_range_bins: int
    n_az_bins: int
    hfov: float                # rad
    vfov: float                # rad
    r_min: float               # m
    r_max: float               # m
    fan_w: int = 0
    fan_h: int = 0

    @property
    def n_rays(self) -> int:
        return self.n_beams * self.n_elev

    def replace_pose(self, pos, rot) -> "SensorSpec":
        s = SensorSpec(**{**self.__dict__})
        s.pos = np.asarray(pos, np.float32).reshape(3)
        s.rot = np.asarray(rot, np.float32).reshape(3, 3)
        return s


# ----------------------------------------------------------------------------
# primitive meshes
# ----------------------------------------------------------------------------

def quad(z: float, half_extent: float, mat_id: int = 0) -> Mesh:
    """Two triangles covering [-e, e]^2 at height z, normal +z."""
    e = float(half_extent)
    v = np.array([[-e, -e, z], [e, -e, z], [e, e, z], [-e, e, z]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return Mesh(v, t, np.full(2, mat_id, np.int32))


def _icosahedron():
    g = (1.0 + math.sqrt(5.0)) / 2.0
    base = []
    for a, b in itertools.product((-1.0, 1.0), repeat=2):
        base += [(0.0, a, b * g), (a, b * g, 0.0), (b * g, 0.0, a)]
    v = np.array(base, np.float64)
    # faces = vertex triples whose three pairwise distances equal the edge length 2
    faces = []
    for i, j, k in itertools.combinations(range(12), 3):
        d = [np.linalg.norm(v[i] - v[j]), np.linalg.norm(v[j] - v[k]), np.linalg.norm(v[i] - v[k])]
        if all(abs(x - 2.0) < 1e-9 for x in d):
            n = np.cross(v[j] - v[i], v[k] - v[i])
            faces.append((i, j, k) if np.dot(n, v[i] + v[j] + v[k]) > 0 else (i, k, j))
    assert len(faces) == 20
    return v / np.linalg.norm(v, axis=1, keepdims=True), faces


def icosphere(subdiv: int, radius: float, center, mat_id: int = 0) -> Mesh:
    """Icosahedron subdivided `subdiv` times (20 * 4^subdiv faces), vertices
    projected onto the sphere; outward winding."""
    v, faces = _icosahedron()
    verts = [tuple(p) for p in v]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                p = (np.array(verts[a]) + np.array(verts[b])) * 0.5
                p /= np.linalg.norm(p)
                cache[key] = len(verts)
                verts.append(tuple(p))
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    p = np.array(verts, np.float64) * radius + np.asarray(center, np.float64)
    return Mesh(p.astype(np.float32), np.array(faces, np.int32),
                np.full(len(faces), mat_id, np.int32))


def _value_noise_fbm(x, y, extent, seed, octaves=6, lacunarity=2.0, persistence=0.5,
                     base_cells=4):
    """fBm of bilinear (smoothstep-weighted) value noise on [-extent/2, extent/2]^2,
    normalised so that the result lies in [-1, 1]."""
    rng = np.random.default_rng(seed)
    u = (np.asarray(x, np.float64) / extent) + 0.5
    w = (np.asarray(y, np.float64) / extent) + 0.5
    total = np.zeros(np.broadcast(u, w).shape)
    norm = 0.0
    amp = 1.0
    cells = float(base_cells)
    for _ in range(octaves):
        n = int(round(cells))
        lattice = rng.uniform(-1.0, 1.0, size=(n + 2, n + 2))
        fu = np.clip(u * n, 0.0, n - 1e-9)
        fw = np.clip(w * n, 0.0, n - 1e-9)
        iu = np.floor(fu).astype(np.int64)
        iw = np.floor(fw).astype(np.int64)
        tu = fu - iu
        tw = fw - iw
        su = tu * tu * (3.0 - 2.0 * tu)
        sw = tw * tw * (3.0 - 2.0 * tw)
        a = lattice[iu, iw]
        b = lattice[iu + 1, iw]
        c = lattice[iu, iw + 1]
        d = lattice[iu + 1, iw + 1]
        total += amp * ((a * (1 - su) + b * su) * (1 - sw) + (c * (1 - su) + d * su) * sw)
        norm += amp
        amp *= persistence
        cells *= lacunarity
    return total / norm


def height_function(extent: float, amplitude: float, seed: int, z0: float = 0.0):
    """The seabed surface z0 + amplitude * fBm(x, y) of a heightfield scene,
    evaluable at arbitrary points without building the mesh."""
    def height_fn(x, y):
        return z0 + amplitude * _value_noise_fbm(x, y, extent, seed)
    return height_fn


def heightfield(n_cells: int, extent: float, amplitude: float, seed: int,
                patches: int = 4, mat_base: int = 0, z0: float = 0.0):
    """Regular n x n cell grid over [-extent/2, extent/2]^2 with heights
    z0 + amplitude * fBm.  Each cell is split along a fixed diagonal into two
    upward-facing triangles (2 n^2 triangles).  Materials: patches x patches
    square patches, ids mat_base .. mat_base + patches^2 - 1.

    Returns (mesh, height_fn) where height_fn(x, y) evaluates the same surface
    at arbitrary points (used to stand obstacles on the seabed)."""
    n = int(n_cells)
    xs = (np.arange(n + 1, dtype=np.float64) / n - 0.5) * extent
    X, Y = np.meshgrid(xs, xs, indexing="ij")          # vertex (i, j) at X[i,j], Y[i,j]
    height_fn = height_function(extent, amplitude, seed, z0)
    Z = height_fn(X, Y)
    verts = np.stack([X, Y, Z], axis=-1).reshape(-1, 3).astype(np.float32)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a = (i * (n + 1) + j).ravel()
    b = ((i + 1) * (n + 1) + j).ravel()
    c = ((i + 1) * (n + 1) + j + 1).ravel()
    d = (i * (n + 1) + j + 1).ravel()
    tris = np.empty((2 * n * n, 3), np.int32)
    tris[0::2] = np.stack([a, b, c], axis=1)
    tris[1::2] = np.stack([a, c, d], axis=1)
    pi = np.minimum(i.ravel() * patches // n, patches - 1)
    pj = np.minimum(j.ravel() * patches // n, patches - 1)
    cell_mat = (mat_base + pi * patches + pj).astype(np.int32)
    mat = np.repeat(cell_mat, 2)
    return Mesh(verts, tris, mat, {"kind": "heightfield", "n_cells": n}), height_fn


def cylinder(center_xy, z_base: float, radius: float, height: float, sides: int = 16,
             mat_id: int = 0) -> Mesh:
    """Closed `sides`-gon prism: 2*sides wall triangles + 2*sides cap triangles."""
    cx, cy = center_xy
    ang = np.arange(sides) * (2.0 * math.pi / sides)
    ring = np.stack([cx + radius * np.cos(ang), cy + radius * np.sin(ang)], axis=1)
    bot = np.concatenate([ring, np.full((sides, 1), z_base)], axis=1)
    top = np.concatenate([ring, np.full((sides, 1), z_base + height)], axis=1)
    verts = np.concatenate([bot, top, [[cx, cy, z_base]], [[cx, cy, z_base + height]]])
    cb, ct = 2 * sides, 2 * sides + 1
    tris = []
    for k in range(sides):
        k1 = (k + 1) % sides
        tris += [(k, k1, sides + k1), (k, sides + k1, sides + k)]   # wall, outward
        tris += [(cb, k1, k)]                                      # bottom cap, -z
        tris += [(ct, sides + k, sides + k1)]                      # top cap, +z
    return Mesh(verts.astype(np.float32), np.array(tris, np.int32),
                np.full(len(tris), mat_id, np.int32))


def box(center_xy, z_base: float, size, yaw: float = 0.0, mat_id: int = 0) -> Mesh:
    """Closed box (12 triangles, outward winding) standing at z_base, rotated by yaw."""
    sx, sy, sz = size
    corners = np.array([[x, y, z] for z in (0.0, sz) for y in (-sy / 2, sy / 2)
                        for x in (-sx / 2, sx / 2)], np.float64)
    c, s = math.cos(yaw), math.sin(yaw)
    rz = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    verts = corners @ rz.T + np.array([center_xy[0], center_xy[1], z_base])
    # corner index = 4*zbit + 2*ybit + xbit
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    tris = []
    for a, b, cc, d in quads:
        tris += [(a, b, cc), (a, cc, d)]
    tri = np.array(tris, np.int32)
    # orient outward: normal must point away from the box centre
    ctr = verts.mean(axis=0)
    for k in range(len(tri)):
        p = verts[tri[k]]
        n = np.cross(p[1] - p[0], p[2] - p[0])
        if np.dot(n, p.mean(axis=0) - ctr) < 0:
            tri[k] = tri[k][[0, 2, 1]]
    return Mesh(verts.astype(np.float32), tri, np.full(len(tri), mat_id, np.int32))


def merge(meshes) -> Mesh:
    verts, tris, mats, off = [], [], [], 0
    for m in meshes:
        verts.append(m.verts)
        tris.append(m.tris + off)
        mats.append(m.mat)
        off += m.verts.shape[0]
    return Mesh(np.ascontiguousarray(np.concatenate(verts), np.float32),
                np.ascontiguousarray(np.concatenate(tris), np.int32),
                np.ascontiguousarray(np.concatenate(mats), np.int32))


def materials_uniform(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=n).astype(np.float32)


# ----------------------------------------------------------------------------
# poses and sensors
# ----------------------------------------------------------------------------

def pose_matrix(yaw: float = 0.0, pitch_down: float = 0.0) -> np.ndarray:
    """Sensor->world rotation: first pitch the sensor down by `pitch_down`
    (a rotation about +x by -pitch_down), then yaw about +z."""
    cp, sp = math.cos(pitch_down), math.sin(pitch_down)
    rx = np.array([[1.0, 0.0, 0.0], [0.0, cp, sp], [0.0, -sp, cp]])
    cy, sy = math.cos(yaw), math.sin(yaw)
    rz = np.array([[cy, -sy, 0.0], [sy, cy, 0.0], [0.0, 0.0, 1.0]])
    return (rz @ rx).astype(np.float32)


def sensor_tiny(pitch_deg: float = 20.0) -> SensorSpec:
    """128 beams over 60 deg x 8 elevation rays over 12 deg, 0.5-10 m, 256 range
    bins x 128 azimuth bins, 400 x 300 fan; at the origin, pitched down."""
    return SensorSpec(np.zeros(3, np.float32), pose_matrix(0.0, math.radians(pitch_deg)),
                      128, 8, 256, 128, math.radians(60.0), math.radians(12.0), 0.5, 10.0,
                      400, 300)


def tiny_scene():
    """Seabed quad (2 tris, z=-5, +-50 m, mu=0.3 as material 0) and a unit
    icosphere (subdiv 3, 1280 tris) at (0, 4, -3.5) (material 1, mu=0.8)."""
    m = merge([quad(-5.0, 50.0, 0), icosphere(3, 1.0, (0.0, 4.0, -3.5), 1)])
    return m, np.array([0.3, 0.8], np.float32)


def single_frame_scene(n_cells=1024, extent=100.0, amplitude=2.0, seed=1, n_piles=48,
                       n_boxes=24, n_mat=16, mu_lo=0.1, mu_hi=0.9, keep_clear=2.0,
                       mu_seed=None):
    """Seabed heightfield plus pier piles and boxes standing on it.
    Returns (mesh, mu[n_mat], height_fn)."""
    patches = int(round(math.sqrt(n_mat)))
    assert patches * patches == n_mat
    hf, hfn = heightfield(n_cells, extent, amplitude, seed, patches=patches)
    rng = np.random.default_rng(seed + 1000)
    parts = [hf]
    half = extent / 2.0 - 5.0

    def place():
        while True:
            x, y = rng.uniform(-half, half, size=2)
            if math.hypot(x, y) > keep_clear + 4.0:
                return float(x), float(y)

    for _ in range(n_piles):
        x, y = place()
        parts.append(cylinder((x, y), float(hfn(x, y)) - 0.5, rng.uniform(0.3, 1.0),
                              rng.uniform(3.0, 8.0), 16, int(rng.integers(0, n_mat))))
    for _ in range(n_boxes):
        x, y = place()
        parts.append(box((x, y), float(hfn(x, y)) - 0.3, rng.uniform(0.5, 4.0, size=3),
                         rng.uniform(0, math.pi), int(rng.integers(0, n_mat))))
    mesh = merge(parts)
    mesh.info = {"kind": "seabed", "n_cells": n_cells, "extent": extent, "seed": seed}
    mu = materials_uniform(n_mat, mu_lo, mu_hi, seed + 2000 if mu_seed is None else mu_seed)
    return mesh, mu, hfn


def large_scene(n_cells=4096, extent=400.0, amplitude=4.0, seed=7, n_obstacles=2000, n_mat=64):
    return single_frame_scene(n_cells, extent, amplitude, seed, n_piles=n_obstacles // 2,
                              n_boxes=n_obstacles - n_obstacles // 2, n_mat=n_mat,
                              mu_lo=0.05, mu_hi=0.95)


def sensor_single(height_fn, altitude=4.0, pitch_deg=25.0, yaw=0.0, xy=(0.0, 0.0),
                  n_beams=512, n_elev=64, n_range_bins=1000, n_az_bins=None,
                  hfov_deg=130.0, vfov_deg=20.0, r_min=0.1, r_max=20.0,
                  fan_w=1024, fan_h=576) -> SensorSpec:
    """The 512 x 64 ray, 1000-bin sonar over the seabed (Oculus M750-d field of view)."""
    x, y = xy
    pos = np.array([x, y, float(height_fn(x, y)) + altitude], np.float32)
    return SensorSpec(pos, pose_matrix(yaw, math.radians(pitch_deg)), n_beams, n_elev,
                      n_range_bins, n_beams if n_az_bins is None else n_az_bins,
                      math.radians(hfov_deg), math.radians(vfov_deg), r_min, r_max,
                      fan_w, fan_h)


def trajectory(base: SensorSpec, height_fn, n_poses: int, radius=20.0, altitude=4.0,
               pitch_deg=25.0, seed=0):
    """Poses on a circle of the given radius, looking along the direction of
    travel, `altitude` above the seabed; small seeded pitch jitter."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_poses):
        a = 2.0 * math.pi * k / n_poses
        x, y = radius * math.cos(a), radius * math.sin(a)
        yaw = a  # tangent of a counter-clockwise circle, in this frame
        pos = (x, y, float(height_fn(x, y)) + altitude)
        pitch = math.radians(pitch_deg + rng.uniform(-2.0, 2.0))
        out.append(base.replace_pose(pos, pose_matrix(yaw, pitch)))
    return out


SENSOR_TYPES = ((256, 32, 500), (512, 64, 1000), (1024, 128, 2000))


def batched_workload(n_sensors=128, seed=11, grids=(512, 640, 768, 1024), extent=100.0,
                     amplitude=2.0, n_mat=16):
    """Four heightfield scenes (seeds 2-5) and `n_sensors` sensors of three
    types on random poses: HFOV U[60,130] deg, VFOV U[12,20] deg, r_max
    U[10,40] m, 2-6 m altitude, pitch 15-35 deg down.
    Returns (scenes[list of (mesh, height_fn)], mu, list of (scene_index, SensorSpec))."""
    scenes = []
    for k, g in enumerate(grids):
        m, mu, hfn = single_frame_scene(n_cells=g, extent=extent, amplitude=amplitude,
                                        seed=2 + k, n_mat=n_mat)
        scenes.append((m, hfn))
    mu = materials_uniform(n_mat, 0.1, 0.9, seed + 3000)
    rng = np.random.default_rng(seed)
    sensors = []
    for _ in range(n_sensors):
        si = int(rng.integers(0, len(scenes)))
        nb, ne, nr = SENSOR_TYPES[int(rng.integers(0, 3))]
        hfn = scenes[si][1]
        x, y = rng.uniform(-35.0, 35.0, size=2)
        alt = rng.uniform(2.0, 6.0)
        s = sensor_single(hfn, altitude=alt, pitch_deg=rng.uniform(15.0, 35.0),
                          yaw=rng.uniform(0, 2 * math.pi), xy=(x, y), n_beams=nb, n_elev=ne,
                          n_range_bins=nr, hfov_deg=rng.uniform(60.0, 130.0),
                          vfov_deg=rng.uniform(12.0, 20.0), r_min=0.1,
                          r_max=rng.uniform(10.0, 40.0), fan_w=2 * nb, fan_h=(9 * 2 * nb) // 16)
        sensors.append((si, s))
    return scenes, mu, sensors


def random_soup(n_tris: int, seed: int, center=(0.0, 6.0, -2.0), spread=4.0,
                degenerate_frac=0.05, sliver_frac=0.05, n_mat=4) -> Mesh:
    """Random triangles in a box in front of a sensor at the origin, with a
    share of degenerate (repeated / collinear vertex) and sliver triangles."""
    rng = np.random.default_rng(seed)
    c = np.asarray(center, np.float64)
    p0 = c + rng.uniform(-spread, spread, size=(n_tris, 3))
    e1 = rng.normal(0.0, 0.8, size=(n_tris, 3))
    e2 = rng.normal(0.0, 0.8, size=(n_tris, 3))
    kind = rng.uniform(size=n_tris)
    deg = kind < degenerate_frac
    sl = (kind >= degenerate_frac) & (kind < degenerate_frac + sliver_frac)
    e2[deg] = e1[deg] * rng.choice([0.0, 0.5, 2.0], size=(int(deg.sum()), 1))
    e2[sl] = e1[sl] * 0.7 + rng.normal(0.0, 1e-3, size=(int(sl.sum()), 3))
    verts = np.stack([p0, p0 + e1, p0 + e2], axis=1).reshape(-1, 3).astype(np.float32)
    tris = np.arange(3 * n_tris, dtype=np.int32).reshape(n_tris, 3)
    mat = rng.integers(0, n_mat, size=n_tris).astype(np.int32)
    return Mesh(verts, tris, mat)


# ----------------------------------------------------------------------------
# camera inputs for the underwater image formation (in-air image and depth)
# ----------------------------------------------------------------------------

def camera_rgb(height: int, width: int, seed: int) -> np.ndarray:
    """A seeded in-air RGB image in [0, 1] ([height, width, 3] float32): one
    value-noise fBm texture per channel, mapped through a logistic."""
    y, x = np.meshgrid(np.linspace(-0.5, 0.5, height), np.linspace(-0.5, 0.5, width), indexing="ij")
    ch = [_value_noise_fbm(x, y, 1.0, seed + 31 * c, octaves=5, base_cells=6) for c in range(3)]
    img = 1.0 / (1.0 + np.exp(-2.5 * np.stack(ch, axis=-1)))
    return img.astype(np.float32)


def camera_seabed_depth(height: int, width: int, hfov_deg=90.0, altitude=4.0, pitch_deg=30.0) -> np.ndarray:
    """Distance along each pixel's ray from a pinhole camera `altitude` above a
    flat seabed, pitched `pitch_deg` down ([height, width] float32, +inf for
    rays that do not reach the seabed)."""
    f = 0.5 * width / math.tan(math.radians(hfov_deg) / 2.0)
    v, u = np.meshgrid(np.arange(height) + 0.5 - height / 2.0, np.arange(width) + 0.5 - width / 2.0,
                       indexing="ij")
    # camera frame: x right, y down, z forward; pitched down about x
    p = math.radians(pitch_deg)
    dz = -(v * math.cos(p) + f * math.sin(p))   # world up component of (u, v, f)
    norm = np.sqrt(u * u + v * v + f * f)
    with np.errstate(divide="ignore"):
        t = np.where(dz < 0.0, altitude * norm / np.maximum(-dz, 1e-30), np.inf)
    return t.astype(np.float32)


# ----------------------------------------------------------------------------
# DVL trajectories
# ----------------------------------------------------------------------------

def dvl_trajectories(height_fn, n_veh: int, n_steps: int, dt: float, seed: int, extent=100.0,
                     alt_lo=0.5, alt_hi=70.0):
    """Seeded vehicles crossing a seabed: straight tracks at 0.5-2 m/s, the
    altitude swinging between alt_lo and alt_hi (so beams leave the DVL's
    window and come back), small pitch and roll oscillations.  Returns poses
    [n_veh, n_steps, 12] (position, sensor->world rotation) and world
    velocities [n_veh, n_steps, 3], float32."""
    rng = np.random.default_rng(seed)
    t = (np.arange(n_steps) * dt)[None, :]
    psi = rng.uniform(0, 2 * math.pi, (n_veh, 1))
    speed = rng.uniform(0.5, 2.0, (n_veh, 1))
    x0 = rng.uniform(-0.35 * extent, 0.35 * extent, (n_veh, 1))
    y0 = rng.uniform(-0.35 * extent, 0.35 * extent, (n_veh, 1))
    w_alt, ph = rng.uniform(0.05, 0.4, (n_veh, 1)), rng.uniform(0, 2 * math.pi, (n_veh, 1))
    w_att = rng.uniform(0.2, 1.0, (n_veh, 1))
    pa, ra = rng.uniform(0.0, 0.15, (n_veh, 1)), rng.uniform(0.0, 0.15, (n_veh, 1))
    a_mid, a_amp = 0.5 * (alt_lo + alt_hi), 0.5 * (alt_hi - alt_lo)
    x = x0 + speed * np.cos(psi) * t
    y = y0 + speed * np.sin(psi) * t
    z = height_fn(x, y) + a_mid + a_amp * np.sin(w_alt * t + ph)
    dz = np.gradient(z, dt, axis=1) if n_steps > 1 else np.zeros_like(z)
    pitch, roll = pa * np.sin(w_att * t), ra * np.cos(w_att * t)
    cy, sy = np.broadcast_to(np.cos(psi), z.shape), np.broadcast_to(np.sin(psi), z.shape)
    cp, sp, cr, sr = np.cos(pitch), np.sin(pitch), np.cos(roll), np.sin(roll)
    # R = Rz(psi) Rx(pitch) Ry(roll), row-major
    R = np.stack([cy * cr - sy * sp * sr, -sy * cp, cy * sr + sy * sp * cr,
                  sy * cr + cy * sp * sr, cy * cp, sy * sr - cy * sp * cr,
                  -cp * sr, sp, cp * cr], axis=-1)
    poses = np.concatenate([np.stack([x, y, z], axis=-1), R], axis=-1)
    vels = np.stack([np.broadcast_to(speed * np.cos(psi), z.shape), np.broadcast_to(speed * np.sin(psi), z.shape),
                     dz], axis=-1)
    return poses.astype(np.float32), vels.astype(np.float32)
