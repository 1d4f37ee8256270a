"""Procedural scene, camera and path sampler for the synthetic vertex streams.

Vertex record (64 bytes, 16 float32, array-of-structures)::

    v0 = (px, py, pz, w)      hit position, MIS weight w
    v1 = (nx, ny, nz, tr)     geometric normal, throughput red
    v2 = (dx, dy, dz, tg)     incoming ray direction (towards the surface), throughput green
    v3 = (Lr, Lg, Lb, tb)     radiance estimate at the vertex, throughput blue

The throughput t = f*cos/p (per channel) is the path-tracer weight carried from
this vertex to the next one (Alg. 1 keeps it as f_j w_j / p_j).  The outgoing
direction of the vertex is omega_o = -d (Alg. 1 sets omega^o_j = -omega^i_{j-1}).
A stream for P paths of depth D holds D*P records in depth-major order:
record j*P + p is the j-th surface hit of path p, and pixel p = y*W + x.

Scene (stands in for the paper's interior scenes, which are not available):
the closed unit box [0,1]^3 (six walls, inward normals) and two spheres of
radius 0.2 with outward normals, centres drawn uniformly in [0.3,0.7]^3 and
redrawn until the spheres do not overlap.  Every surface is Lambertian with a
per-object RGB albedo rho ~ lognormal(0, 0.5) clamped to 0.95, so under
cosine-weighted sampling the throughput equals rho exactly.  A pinhole camera
looks along +z (up +y, vertical field of view 60 degrees) from
(camera_x, 0.5, 0.02); every pixel is jittered by U[-0.5, 0.5]^2 each
iteration.  Every bounce is cosine-distributed about the geometric normal
(Malley's method), the new ray starting 1e-4 along the normal.  The box is
closed, so every path has exactly D surface hits.

Randomness: numpy's Philox4x32 bit generator seeded by SeedSequence
([seed, iteration, stream]), where stream separates the scene, the camera
jitter, the bounce directions and the radiance draws.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FLOATS_PER_VERTEX = 16

_STREAM_SCENE = 0
_STREAM_CAMERA = 1
_STREAM_BOUNCE = 2
_STREAM_RADIANCE = 3
_STREAM_SESSIONS = 4
_STREAM_ARRIVALS = 5

# key-light direction whose mirror image about the normal centres the glossy lobe
_KEY_LIGHT = np.array([0.2, 1.0, 0.4]) / math.sqrt(0.2 ** 2 + 1.0 + 0.4 ** 2)
_GLOSS_EXPONENT = 32


def _rng(seed: int, iteration: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, iteration, stream])))


@dataclass
class Scene:
    sphere_centre: np.ndarray  # (2, 3)
    sphere_radius: float
    albedo: np.ndarray  # (8, 3): walls x0, x1, y0, y1, z0, z1, then the two spheres
    normals: np.ndarray = field(init=False)

    def __post_init__(self):
        n = np.zeros((6, 3))
        for axis in range(3):
            n[2 * axis, axis] = 1.0  # wall at coordinate 0 faces +axis
            n[2 * axis + 1, axis] = -1.0  # wall at coordinate 1 faces -axis
        self.normals = n


def make_scene(seed: int) -> Scene:
    rng = _rng(seed, 0, _STREAM_SCENE)
    r = 0.2
    while True:
        c = rng.uniform(0.3, 0.7, size=(2, 3))
        if np.linalg.norm(c[0] - c[1]) > 2.0 * r + 1e-3:
            break
    albedo = np.minimum(rng.lognormal(0.0, 0.5, size=(8, 3)), 0.95)
    return Scene(sphere_centre=c, sphere_radius=r, albedo=albedo)


def _intersect(scene: Scene, o: np.ndarray, d: np.ndarray):
    """Closest hit of rays (o, d) with the box walls and the spheres.

    Returns (t, object id, hit position, geometric normal)."""
    n_rays = o.shape[0]
    with np.errstate(divide="ignore", invalid="ignore"):
        # the box is closed: the exit face along each axis is the wall hit on that axis
        t_hi = (1.0 - o) / d
        t_lo = (0.0 - o) / d
    t_axis = np.where(d > 0, t_hi, np.where(d < 0, t_lo, np.inf))
    axis = np.argmin(t_axis, axis=1)
    t = t_axis[np.arange(n_rays), axis]
    obj = 2 * axis + (d[np.arange(n_rays), axis] > 0)
    for s in range(2):
        oc = o - scene.sphere_centre[s]
        b = np.einsum("ij,ij->i", oc, d)
        cc = np.einsum("ij,ij->i", oc, oc) - scene.sphere_radius ** 2
        disc = b * b - cc
        ok = disc >= 0
        ts = np.where(ok, -b - np.sqrt(np.where(ok, disc, 0.0)), np.inf)
        hit = (ts > 1e-9) & (ts < t)
        t = np.where(hit, ts, t)
        obj = np.where(hit, 6 + s, obj)
    p = o + t[:, None] * d
    normal = np.empty_like(p)
    wall = obj < 6
    normal[wall] = scene.normals[obj[wall]]
    # put wall hits exactly on their plane
    w_idx = np.nonzero(wall)[0]
    w_axis = obj[w_idx] // 2
    p[w_idx, w_axis] = (obj[w_idx] % 2).astype(np.float64)
    for s in range(2):
        m = obj == 6 + s
        if np.any(m):
            v = p[m] - scene.sphere_centre[s]
            normal[m] = v / np.linalg.norm(v, axis=1, keepdims=True)
    return t, obj, p, normal


def _cosine_about(normal: np.ndarray, u1: np.ndarray, u2: np.ndarray) -> np.ndarray:
    """Cosine-distributed directions about unit normals (Malley's method).

    The tangent frame is the branchless orthonormal basis of Duff et al.,
    "Building an Orthonormal Basis, Revisited" (JCGT 2017)."""
    nx, ny, nz = normal[:, 0], normal[:, 1], normal[:, 2]
    sign = np.where(nz >= 0, 1.0, -1.0)
    a = -1.0 / (sign + nz)
    b = nx * ny * a
    t1 = np.stack([1.0 + sign * nx * nx * a, sign * b, -sign * nx], axis=1)
    t2 = np.stack([b, sign + ny * ny * a, -ny], axis=1)
    r = np.sqrt(u1)
    phi = 2.0 * math.pi * u2
    lx, ly = r * np.cos(phi), r * np.sin(phi)
    lz = np.sqrt(np.maximum(0.0, 1.0 - u1))
    d = lx[:, None] * t1 + ly[:, None] * t2 + lz[:, None] * normal
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def trace_paths(scene: Scene, width: int, height: int, depth: int, *, seed: int, iteration: int,
                camera_x: float = 0.5, radiance: str = "glossy") -> np.ndarray:
    """Trace width*height paths of `depth` surface hits; returns (depth*P, 16) float32."""
    P = width * height
    cam_rng = _rng(seed, iteration, _STREAM_CAMERA)
    bounce_rng = _rng(seed, iteration, _STREAM_BOUNCE)
    rad_rng = _rng(seed, iteration, _STREAM_RADIANCE)

    px = np.tile(np.arange(width, dtype=np.float64), height)
    py = np.repeat(np.arange(height, dtype=np.float64), width)
    jitter = cam_rng.uniform(-0.5, 0.5, size=(P, 2))
    tan_half = math.tan(math.radians(30.0))
    sx = ((px + 0.5 + jitter[:, 0]) / width * 2.0 - 1.0) * tan_half * (width / height)
    sy = (1.0 - (py + 0.5 + jitter[:, 1]) / height * 2.0) * tan_half
    d = np.stack([sx, sy, np.ones(P)], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.tile(np.array([camera_x, 0.5, 0.02]), (P, 1))

    out = np.empty((depth * P, FLOATS_PER_VERTEX), dtype=np.float32)
    for j in range(depth):
        _, obj, p, n = _intersect(scene, o, d)
        rho = scene.albedo[obj]
        if radiance == "lognormal":
            L = rad_rng.lognormal(0.0, 1.0, size=(P, 3))
        elif radiance == "glossy":
            m = 2.0 * (n @ _KEY_LIGHT)[:, None] * n - _KEY_LIGHT
            cos_m = np.maximum(0.0, -np.einsum("ij,ij->i", d, m))
            L = rad_rng.lognormal(0.0, 0.5, size=(P, 3)) * (cos_m ** _GLOSS_EXPONENT)[:, None]
        else:
            raise ValueError(f"unknown radiance model {radiance!r}")
        rec = out[j * P:(j + 1) * P]
        rec[:, 0:3] = p
        rec[:, 3] = 1.0
        rec[:, 4:7] = n
        rec[:, 7] = rho[:, 0]
        rec[:, 8:11] = d
        rec[:, 11] = rho[:, 1]
        rec[:, 12:15] = L
        rec[:, 15] = rho[:, 2]
        if j + 1 < depth:
            u = bounce_rng.random(size=(P, 2))
            o = p + 1e-4 * n
            d = _cosine_about(n, u[:, 0], u[:, 1])
    return out


# ---------------------------------------------------------------------------
# Workload definitions
# ---------------------------------------------------------------------------

def config4_q_bits(log2_capacity: int, dir_bits: int = 3) -> int:
    """Largest q with 7 * 4^q * (4^d / 2) * 1.2 <= capacity / 2 (at least 1).

    7 * 4^q approximates the surface cells of six walls plus the spheres at
    cell size 2^-q, 4^d / 2 the populated half of the 2^d x 2^d direction grid,
    1.2 a margin; the bound keeps the table at most half full."""
    q = 1
    while 7 * 4 ** (q + 1) * (4 ** dir_bits / 2) * 1.2 <= (1 << log2_capacity) / 2:
        q += 1
    return q


_WORKLOADS = {
    "64x64_d3": dict(width=64, height=64, depth=3, iterations=8, log2_capacity=16, pos_bits=4,
                     dir_bits=2, alpha_min=0.1, radiance="lognormal", seed=1, camera_step=0.0,
                     camera_x0=0.5, cache_fp16=False),
    "1280x720_d4": dict(width=1280, height=720, depth=4, iterations=32, log2_capacity=22, pos_bits=6,
                        dir_bits=3, alpha_min=0.1, radiance="glossy", seed=2, camera_step=0.0,
                        camera_x0=0.5, cache_fp16=False),
    "1920x1080_d5": dict(width=1920, height=1080, depth=5, iterations=64, log2_capacity=24, pos_bits=7,
                         dir_bits=3, alpha_min=0.1, radiance="glossy", seed=3, camera_step=0.01,
                         camera_x0=0.18, cache_fp16=True),
}


def workload(name: str) -> dict:
    """Parameters of a named single-session workload (copy)."""
    w = dict(_WORKLOADS[name])
    w["name"] = name
    w["vertices"] = w["width"] * w["height"] * w["depth"]
    return w


def camera_x(w: dict, iteration: int) -> float:
    return w["camera_x0"] + w["camera_step"] * iteration


def session_workloads(n_sessions: int = 64, seed: int = 4, first_session_seed: int = 4000,
                      iterations: int = 32) -> list[dict]:
    """Uneven render sessions: image width log-uniform in [128, 1280], 16:9,
    depth uniform in 2..6, table 2^(ceil(log2 V) + 1) slots, q by config4_q_bits."""
    rng = _rng(seed, 0, _STREAM_SESSIONS)
    out = []
    for s in range(n_sessions):
        wdt = int(round(math.exp(rng.uniform(math.log(128), math.log(1280)))))
        hgt = int(round(9 * wdt / 16))
        dep = int(rng.integers(2, 7))
        v = wdt * hgt * dep
        log2_cap = int(math.ceil(math.log2(v))) + 1
        out.append(dict(name=f"session{s}", width=wdt, height=hgt, depth=dep, iterations=iterations,
                        log2_capacity=log2_cap, pos_bits=config4_q_bits(log2_cap, 3), dir_bits=3,
                        alpha_min=0.1, radiance="glossy", seed=first_session_seed + s,
                        camera_step=0.0, camera_x0=0.5, cache_fp16=True, vertices=v))
    return out


def serving_arrivals(rate_per_s: float, duration_s: float, seed: int = 5) -> list[dict]:
    """Poisson arrivals of render sessions: each lasts U{16..128} iterations and
    draws its size and depth like `session_workloads`."""
    rng = _rng(seed, int(rate_per_s), _STREAM_ARRIVALS)
    t = 0.0
    out = []
    k = 0
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            break
        wdt = int(round(math.exp(rng.uniform(math.log(128), math.log(1280)))))
        hgt = int(round(9 * wdt / 16))
        dep = int(rng.integers(2, 7))
        v = wdt * hgt * dep
        log2_cap = int(math.ceil(math.log2(v))) + 1
        out.append(dict(name=f"req{k}", arrival_s=t, width=wdt, height=hgt, depth=dep,
                        iterations=int(rng.integers(16, 129)), log2_capacity=log2_cap,
                        pos_bits=config4_q_bits(log2_cap, 3), dir_bits=3, alpha_min=0.1,
                        radiance="glossy", seed=10000 + k, camera_step=0.0, camera_x0=0.5,
                        cache_fp16=True, vertices=v))
        k += 1
    return out


def iteration_vertices(w: dict, iteration: int, scene: Scene | None = None) -> np.ndarray:
    """The vertex stream of workload `w` at `iteration`."""
    if scene is None:
        scene = make_scene(w["seed"])
    return trace_paths(scene, w["width"], w["height"], w["depth"], seed=w["seed"], iteration=iteration,
                       camera_x=camera_x(w, iteration), radiance=w["radiance"])
