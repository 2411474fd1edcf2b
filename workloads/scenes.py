"""Seeded triangle scenes shaped like the paper's ray-casting workloads.

The paper measures on Bistro and Sun Temple (Sec. 5.2.1; the Temple has
606,376 triangles).  Those assets are not available, so these procedural
scenes stand in for them at 1K, ~1.07M and ~2.0M triangles.

A scene is a float32 array ``tris`` of shape (n, 3, 3) (triangle, vertex,
xyz), a float32 ``albedo`` of shape (n, 3) in [0.2, 1], and a unit float32
``light_dir`` (direction the light travels).
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Scene:
    tris: np.ndarray      # (n, 3, 3) float32
    albedo: np.ndarray    # (n, 3) float32
    light_dir: np.ndarray  # (3,) float32, unit, direction of light travel
    name: str = ""

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


def _unit(v) -> np.ndarray:
    v = np.asarray(v, dtype=np.float64)
    return (v / np.linalg.norm(v)).astype(np.float32)


DEFAULT_LIGHT = (-0.4, -1.0, 0.6)


def random_triangles_scene(n: int = 1024, seed: int = 1001) -> Scene:
    """n triangles with every vertex uniform in [-1, 1]^3."""
    rng = np.random.default_rng(seed)
    tris = rng.uniform(-1.0, 1.0, size=(n, 3, 3)).astype(np.float32)
    albedo = rng.uniform(0.2, 1.0, size=(n, 3)).astype(np.float32)
    return Scene(tris, albedo, _unit(DEFAULT_LIGHT), f"random{n}")


def tiny_scene(kind: str, seed: int = 7) -> Scene:
    """Hand-placed small scenes for edge cases (all in front of a camera at z=-3)."""
    rng = np.random.default_rng(seed)
    if kind == "empty":
        tris = np.zeros((0, 3, 3), np.float32)
    elif kind == "single":
        tris = np.array([[[-1, -1, 0], [1, -1, 0], [0, 1, 0]]], np.float32)
    elif kind == "quad":
        # two triangles sharing the diagonal edge; rays through the diagonal
        # must hit exactly one of them (no crack)
        a, b, c, d = [-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0]
        tris = np.array([[a, b, c], [a, c, d]], np.float32)
    elif kind == "fan":
        # 8 triangles around a shared centre vertex on the optical axis
        ang = np.linspace(0, 2 * np.pi, 9)[:-1]
        ring = np.stack([np.cos(ang), np.sin(ang), np.zeros_like(ang)], 1)
        tris = np.array([[[0, 0, 0], ring[i], ring[(i + 1) % 8]] for i in range(8)],
                        np.float32)
    elif kind == "stack":
        # coplanar duplicates and parallel layers: exercises the tie rule
        base = np.array([[-1, -1, 0], [1, -1, 0], [0, 1, 0]], np.float32)
        tris = np.stack([base, base, base + [0, 0, 0.5], base[::-1].copy()], 0)
    elif kind == "axis":
        # axis-aligned triangles whose edges lie on pixel rows / columns
        tris = np.array([[[-1, 0, 0], [1, 0, 0], [1, 1, 0]],
                         [[-1, 0, 0], [1, 1, 0], [-1, 1, 0]],
                         [[0, -1, 0.25], [0, 1, 0.25], [1, -1, 0.25]]], np.float32)
    else:
        raise ValueError(kind)
    n = tris.shape[0]
    albedo = rng.uniform(0.2, 1.0, size=(n, 3)).astype(np.float32)
    return Scene(np.ascontiguousarray(tris.reshape(n, 3, 3), dtype=np.float32), albedo,
                 _unit(DEFAULT_LIGHT), f"tiny-{kind}")


# --------------------------------------------------------------------------
# procedural terrain (fBm value noise) + instanced boxes / spheres

def _value_noise(x: np.ndarray, z: np.ndarray, lattice: np.ndarray) -> np.ndarray:
    """Quintic-interpolated value noise on a periodic random lattice."""
    n = lattice.shape[0]
    xi = np.floor(x).astype(np.int64)
    zi = np.floor(z).astype(np.int64)
    fx = x - xi
    fz = z - zi
    sx = fx * fx * fx * (fx * (fx * 6 - 15) + 10)
    sz = fz * fz * fz * (fz * (fz * 6 - 15) + 10)
    x0, x1 = xi % n, (xi + 1) % n
    z0, z1 = zi % n, (zi + 1) % n
    a = lattice[x0, z0]
    b = lattice[x1, z0]
    c = lattice[x0, z1]
    d = lattice[x1, z1]
    return (a * (1 - sx) + b * sx) * (1 - sz) + (c * (1 - sx) + d * sx) * sz


def fbm_heightfield(nx: int, nz: int, extent_x: float, extent_z: float,
                    amplitude: float, seed: int, octaves: int = 6,
                    lacunarity: float = 2.0, gain: float = 0.5,
                    base_period: float = 80.0) -> np.ndarray:
    """Heights (nz, nx) in metres; fBm of value noise (6 octaves by default)."""
    rng = np.random.default_rng(seed)
    xs = np.linspace(-extent_x / 2, extent_x / 2, nx)
    zs = np.linspace(-extent_z / 2, extent_z / 2, nz)
    X, Z = np.meshgrid(xs, zs)
    h = np.zeros_like(X)
    freq, amp, norm = 1.0 / base_period, 1.0, 0.0
    for _ in range(octaves):
        lattice = rng.uniform(-1.0, 1.0, size=(256, 256))
        h += amp * _value_noise(X * freq + 17.0, Z * freq + 31.0, lattice)
        norm += amp
        freq *= lacunarity
        amp *= gain
    return (h / norm * amplitude).astype(np.float64)


def _grid_triangles(h: np.ndarray, extent_x: float, extent_z: float) -> np.ndarray:
    nz, nx = h.shape
    xs = np.linspace(-extent_x / 2, extent_x / 2, nx)
    zs = np.linspace(-extent_z / 2, extent_z / 2, nz)
    X, Z = np.meshgrid(xs, zs)
    V = np.stack([X, h, Z], -1)  # (nz, nx, 3)
    a = V[:-1, :-1].reshape(-1, 3)
    b = V[:-1, 1:].reshape(-1, 3)
    c = V[1:, 1:].reshape(-1, 3)
    d = V[1:, :-1].reshape(-1, 3)
    t1 = np.stack([a, b, c], 1)
    t2 = np.stack([a, c, d], 1)
    return np.stack([t1, t2], 1).reshape(-1, 3, 3)


def _height_at(h: np.ndarray, extent_x: float, extent_z: float, x, z):
    nz, nx = h.shape
    fx = (np.asarray(x) + extent_x / 2) / extent_x * (nx - 1)
    fz = (np.asarray(z) + extent_z / 2) / extent_z * (nz - 1)
    ix = np.clip(np.round(fx).astype(np.int64), 0, nx - 1)
    iz = np.clip(np.round(fz).astype(np.int64), 0, nz - 1)
    return h[iz, ix]


_BOX_FACES = np.array([
    [0, 1, 2], [0, 2, 3], [4, 6, 5], [4, 7, 6], [0, 4, 5], [0, 5, 1],
    [1, 5, 6], [1, 6, 2], [2, 6, 7], [2, 7, 3], [3, 7, 4], [3, 4, 0]])


def _unit_box() -> np.ndarray:
    c = np.array([[-1, 0, -1], [1, 0, -1], [1, 0, 1], [-1, 0, 1],
                  [-1, 2, -1], [1, 2, -1], [1, 2, 1], [-1, 2, 1]], np.float64) * 0.5
    return c[_BOX_FACES]  # (12, 3, 3), base on y=0, height 1


def _unit_sphere(slices: int = 8, stacks: int = 5) -> np.ndarray:
    """UV sphere of radius 0.5 resting on y=0: 2*slices*(stacks-1) triangles (64)."""
    tris = []
    th = np.linspace(0, np.pi, stacks + 1)
    ph = np.linspace(0, 2 * np.pi, slices + 1)

    def p(i, j):
        return np.array([np.sin(th[i]) * np.cos(ph[j]), np.cos(th[i]) + 1.0,
                         np.sin(th[i]) * np.sin(ph[j])]) * 0.5
    for i in range(stacks):
        for j in range(slices):
            a, b, c, d = p(i, j), p(i, j + 1), p(i + 1, j + 1), p(i + 1, j)
            if i == 0:
                tris.append([a, c, d])
            elif i == stacks - 1:
                tris.append([a, b, c])
            else:
                tris.append([a, b, c])
                tris.append([a, c, d])
    return np.array(tris)


def _instances(proto: np.ndarray, n: int, rng, h, ex, ez, smin, smax) -> np.ndarray:
    px = rng.uniform(-ex / 2 * 0.95, ex / 2 * 0.95, n)
    pz = rng.uniform(-ez / 2 * 0.95, ez / 2 * 0.95, n)
    s = rng.uniform(smin, smax, n)
    yaw = rng.uniform(0, 2 * np.pi, n)
    py = _height_at(h, ex, ez, px, pz) - 0.1 * s
    cy, sy = np.cos(yaw), np.sin(yaw)
    R = np.zeros((n, 3, 3))
    R[:, 0, 0], R[:, 0, 2], R[:, 1, 1], R[:, 2, 0], R[:, 2, 2] = cy, sy, 1.0, -sy, cy
    P = proto[None] * s[:, None, None, None]             # (n, k, 3, 3)
    P = np.einsum("nij,nkvj->nkvi", R, P)
    P += np.stack([px, py, pz], 1)[:, None, None, :]
    return P.reshape(-1, 3, 3)


def terrain_boxes_scene(nx: int = 512, nz: int = 1024, n_boxes: int = 2000,
                        seed: int = 1002) -> Scene:
    """fBm terrain (nx x nz vertices over 200 m x 400 m, 20 m amplitude) plus
    n_boxes instanced boxes (12 triangles each).  Default: 1,069,506 triangles."""
    ex, ez = 200.0, 400.0
    rng = np.random.default_rng(seed)
    h = fbm_heightfield(nx, nz, ex, ez, 20.0, seed=seed + 1)
    terr = _grid_triangles(h, ex, ez)
    boxes = _instances(_unit_box(), n_boxes, rng, h, ex, ez, 1.0, 8.0)
    tris = np.concatenate([terr, boxes], 0).astype(np.float32)
    alb_t = np.clip(np.array([0.35, 0.55, 0.25]) + rng.normal(0, 0.05, (len(terr), 3)),
                    0.2, 1.0)
    alb_b = np.repeat(rng.uniform(0.2, 1.0, (n_boxes, 3)), 12, 0)
    albedo = np.concatenate([alb_t, alb_b], 0).astype(np.float32)
    scene = Scene(tris, albedo, _unit(DEFAULT_LIGHT), f"terrain{nx}x{nz}+{n_boxes}boxes")
    scene.heights = h  # used to place cameras above the ground
    scene.extent = (ex, ez)
    return scene


def terrain_objects_scene(nx: int = 829, nz: int = 1024, n_spheres: int = 4000,
                          n_boxes: int = 4000, seed: int = 1003) -> Scene:
    """Terrain plus 64-triangle spheres and 12-triangle boxes.
    Default: 1,694,088 + 256,000 + 48,000 = 1,998,088 triangles."""
    ex, ez = 200.0, 400.0
    rng = np.random.default_rng(seed)
    h = fbm_heightfield(nx, nz, ex, ez, 20.0, seed=seed + 1)
    terr = _grid_triangles(h, ex, ez)
    sph = _instances(_unit_sphere(), n_spheres, rng, h, ex, ez, 1.0, 6.0)
    box = _instances(_unit_box(), n_boxes, rng, h, ex, ez, 1.0, 8.0)
    tris = np.concatenate([terr, sph, box], 0).astype(np.float32)
    alb_t = np.clip(np.array([0.35, 0.55, 0.25]) + rng.normal(0, 0.05, (len(terr), 3)),
                    0.2, 1.0)
    alb_s = np.repeat(rng.uniform(0.2, 1.0, (n_spheres, 3)), 64, 0)
    alb_b = np.repeat(rng.uniform(0.2, 1.0, (n_boxes, 3)), 12, 0)
    albedo = np.concatenate([alb_t, alb_s, alb_b], 0).astype(np.float32)
    scene = Scene(tris, albedo, _unit(DEFAULT_LIGHT),
                  f"terrain{nx}x{nz}+{n_spheres}spheres+{n_boxes}boxes")
    scene.heights = h
    scene.extent = (ex, ez)
    return scene
