"""Seeded synthetic triangle meshes for the Monte Carlo DtN estimator.

This module builds INPUTS only: vertex and face arrays of closed (or nearly
closed) surfaces with the shape statistics of the paper's workloads.  It holds
none of the estimator's arithmetic (no normals, areas, sampling, walks or
operators); both the CUDA path and the CPU oracle consume what it returns.

Workloads (the paper's in-the-wild meshes come from Thingi10k / Objaverse,
which are not available offline; these generators stand in for them):

* ``icosphere(s)``           -- unit sphere, icosahedron split 4-way s times.
* ``two_spheres(s, R, D)``   -- two disjoint icospheres, radius R, centres D apart
                               along x (the first centred at the origin).
* ``wild_union(...)``        -- union of random ellipsoids and tori with
                               log-uniform scales, random rotations, vertex noise,
                               a fraction of flipped faces and sliver tessellations
                               (multi-component, overlapping and disjoint), the
                               "in the wild" geometry of the paper's Sec. 5-6
                               (moose 2M faces, Commodore 64, sliver CAD model).
* ``batch_meshes(n, ...)``   -- many wild meshes of uneven size for the batched
                               launch (the Objaverse-scale preprocessing of Sec. 6).

All arrays: V float64 (nv, 3) C-contiguous, F int32 (nf, 3) C-contiguous.
"""
from __future__ import annotations

import math
import numpy as np

__all__ = ["icosphere", "two_spheres", "wild_union", "batch_meshes", "Mesh"]


class Mesh:
    """A plain (V, F) pair with an optional note about how it was made."""

    def __init__(self, V: np.ndarray, F: np.ndarray, note: str = ""):
        self.V = np.ascontiguousarray(V, dtype=np.float64)
        self.F = np.ascontiguousarray(F, dtype=np.int32)
        self.note = note

    @property
    def nv(self) -> int:
        return int(self.V.shape[0])

    @property
    def nf(self) -> int:
        return int(self.F.shape[0])

    def __repr__(self) -> str:
        return f"Mesh(nv={self.nv}, nf={self.nf}, {self.note})"


def _orient_outward(V: np.ndarray, F: np.ndarray, center: np.ndarray) -> np.ndarray:
    """Flip faces of a star-shaped surface so that they wind counter-clockwise
    seen from outside (used only while constructing the inputs)."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    nrm = np.cross(b - a, c - a)
    out = ((a + b + c) / 3.0 - center)
    flip = np.einsum("ij,ij->i", nrm, out) < 0
    F = F.copy()
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return F


def icosphere(subdiv: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)) -> Mesh:
    """Icosahedron split 4-way ``subdiv`` times, vertices pushed to the sphere.

    V = 10*4^s + 2, F = 20*4^s (s=2: 162/320, s=4: 2562/5120)."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, phi, 0), (1, phi, 0), (-1, -phi, 0), (1, -phi, 0),
             (0, -1, phi), (0, 1, phi), (0, -1, -phi), (0, 1, -phi),
             (phi, 0, -1), (phi, 0, 1), (-phi, 0, -1), (-phi, 0, 1)]
    V = [np.array(v, dtype=np.float64) / math.sqrt(1.0 + phi * phi) for v in verts]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        mid = {}
        newF = []

        def midpoint(i, j):
            key = (i, j) if i < j else (j, i)
            k = mid.get(key)
            if k is None:
                m = V[i] + V[j]
                V.append(m / np.linalg.norm(m))
                k = len(V) - 1
                mid[key] = k
            return k

        for (i, j, k) in F:
            a = midpoint(i, j)
            b = midpoint(j, k)
            c = midpoint(k, i)
            newF += [(i, a, c), (j, b, a), (k, c, b), (a, b, c)]
        F = newF
    Va = np.array(V) * radius + np.asarray(center, dtype=np.float64)
    Fa = _orient_outward(Va, np.array(F, dtype=np.int64), np.asarray(center, dtype=np.float64))
    return Mesh(Va, Fa, f"icosphere s{subdiv} R={radius}")


def two_spheres(subdiv: int = 4, radius: float = 0.5, sep: float = 1.5) -> Mesh:
    """Two icospheres of radius ``radius``; centres (0,0,0) and (sep,0,0)."""
    A = icosphere(subdiv, radius, (0.0, 0.0, 0.0))
    B = icosphere(subdiv, radius, (sep, 0.0, 0.0))
    V = np.concatenate([A.V, B.V])
    F = np.concatenate([A.F, B.F + A.nv])
    return Mesh(V, F, f"two icospheres s{subdiv} R={radius} D={sep}")


# ----------------------------------------------------------------------------
# in-the-wild unions
# ----------------------------------------------------------------------------

def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a uniform unit quaternion (Shoemake 1992)."""
    u1, u2, u3 = rng.random(3)
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
                  math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3),
                  math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _uv_ellipsoid(axes, n_lat: int, n_lon: int):
    """Latitude/longitude ellipsoid: 2 poles + n_lat rings of n_lon vertices;
    F = 2 * n_lon * n_lat."""
    a, b, c = axes
    th = np.pi * np.arange(1, n_lat + 1) / (n_lat + 1)
    ph = 2 * np.pi * np.arange(n_lon) / n_lon
    T, P = np.meshgrid(th, ph, indexing="ij")
    ring = np.stack([a * np.sin(T) * np.cos(P), b * np.sin(T) * np.sin(P), c * np.cos(T)], -1)
    V = np.concatenate([[[0, 0, c]], ring.reshape(-1, 3), [[0, 0, -c]]])
    J = np.arange(n_lon)
    Jn = (J + 1) % n_lon
    top = np.stack([np.zeros(n_lon, np.int64), 1 + J, 1 + Jn], -1)
    I = np.arange(n_lat - 1)[:, None]
    q00 = 1 + I * n_lon + J[None, :]
    q01 = 1 + I * n_lon + Jn[None, :]
    q10 = q00 + n_lon
    q11 = q01 + n_lon
    mid1 = np.stack([q00, q10, q11], -1).reshape(-1, 3)
    mid2 = np.stack([q00, q11, q01], -1).reshape(-1, 3)
    sp = 1 + n_lat * n_lon
    bot = np.stack([np.full(n_lon, sp), 1 + (n_lat - 1) * n_lon + Jn, 1 + (n_lat - 1) * n_lon + J], -1)
    F = np.concatenate([top, mid1, mid2, bot]).astype(np.int64)
    return V, _orient_outward(V, F, np.zeros(3))


def _uv_torus(R0: float, r0: float, nu: int, nv: int):
    """Torus around z: major radius R0, tube radius r0; F = 2 * nu * nv."""
    u = 2 * np.pi * np.arange(nu) / nu
    v = 2 * np.pi * np.arange(nv) / nv
    U, Vv = np.meshgrid(u, v, indexing="ij")
    X = np.stack([(R0 + r0 * np.cos(Vv)) * np.cos(U), (R0 + r0 * np.cos(Vv)) * np.sin(U), r0 * np.sin(Vv)], -1)
    V = X.reshape(-1, 3)
    idx = lambda i, j: (i % nu) * nv + (j % nv)
    I, J = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    I, J = I.ravel(), J.ravel()
    F1 = np.stack([idx(I, J), idx(I + 1, J), idx(I + 1, J + 1)], -1)
    F2 = np.stack([idx(I, J), idx(I + 1, J + 1), idx(I, J + 1)], -1)
    F = np.concatenate([F1, F2]).astype(np.int64)
    # orient: outward from the tube's centre circle
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    cen = (a + b + c) / 3.0
    ring = cen.copy()
    ring[:, 2] = 0
    rn = np.linalg.norm(ring, axis=1, keepdims=True)
    ring = ring / np.maximum(rn, 1e-300) * R0
    nrm = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", nrm, cen - ring) < 0
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return V, F


def _ellipsoid_area(a, b, c):
    p = 1.6075  # Knud Thomsen's approximation, |err| < 1.1%
    return 4 * np.pi * (((a * b) ** p + (a * c) ** p + (b * c) ** p) / 3.0) ** (1.0 / p)


def wild_union(n_prims: int = 300, target_faces: int = 2_000_000, seed: int = 0,
               noise: float = 1e-3, flip_frac: float = 0.05, sliver_frac: float = 0.10,
               min_faces: int = 200, scale_range=(0.01, 1.0)) -> Mesh:
    """Union of random ellipsoids (60%) and tori (40%).

    Scales s ~ log-uniform(scale_range); ellipsoid semi-axes s*U[0.3,1]^3,
    torus major radius s and tube radius s*U[0.1,0.4]; centres U[-1,1]^3;
    uniform random rotations; faces allocated in proportion to area (at least
    ``min_faces`` each); vertex noise N(0, noise^2); ``flip_frac`` of faces
    reversed; ``sliver_frac`` of primitives tessellated with aspect >= 20."""
    rng = np.random.default_rng(seed)
    kinds = rng.random(n_prims) < 0.6  # True: ellipsoid
    lo, hi = np.log(scale_range[0]), np.log(scale_range[1])
    scales = np.exp(rng.uniform(lo, hi, n_prims))
    shape_par = rng.uniform(0.3, 1.0, (n_prims, 3))
    tube = rng.uniform(0.1, 0.4, n_prims)
    centres = rng.uniform(-1.0, 1.0, (n_prims, 3))
    sliver = rng.random(n_prims) < sliver_frac
    rots = [_random_rotation(rng) for _ in range(n_prims)]
    areas = np.where(kinds, _ellipsoid_area(*(scales[:, None] * shape_par).T),
                     4 * np.pi ** 2 * scales * (scales * tube))
    alloc = np.maximum(min_faces, np.round(target_faces * areas / areas.sum())).astype(np.int64)
    Vs, Fs, off = [], [], 0
    for p in range(n_prims):
        nf = int(alloc[p])
        if kinds[p]:
            axes = scales[p] * shape_par[p]
            if sliver[p]:
                n_lat = max(2, int(round(math.sqrt(nf / 80.0))))
                n_lon = max(40 * (n_lat + 1), nf // (2 * n_lat))
            else:
                n_lat = max(2, int(round(math.sqrt(nf / 4.0))))
                n_lon = max(3, nf // (2 * n_lat))
            V, F = _uv_ellipsoid(axes, n_lat, n_lon)
        else:
            R0, r0 = scales[p], scales[p] * tube[p]
            ratio = R0 / r0
            if sliver[p]:
                nv_ = max(3, int(round(math.sqrt(nf / (2.0 * 20.0 * ratio)))))
                nu_ = max(int(math.ceil(20 * ratio * nv_)), nf // (2 * nv_))
            else:
                nv_ = max(3, int(round(math.sqrt(nf / (2.0 * ratio)))))
                nu_ = max(3, nf // (2 * nv_))
            V, F = _uv_torus(R0, r0, nu_, nv_)
        V = V @ rots[p].T + centres[p]
        Vs.append(V)
        Fs.append(F + off)
        off += V.shape[0]
    V = np.concatenate(Vs)
    F = np.concatenate(Fs)
    V = V + rng.normal(0.0, noise, V.shape)
    nflip = int(round(flip_frac * F.shape[0]))
    flip = rng.choice(F.shape[0], nflip, replace=False)
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return Mesh(V, F, f"wild union n_prims={n_prims} seed={seed}")


def batch_mesh_params(i: int, seed0: int = 1000, faces_range=(5_000, 200_000), prims_range=(1, 50)):
    """(faces, primitives, min_faces) of mesh i of a batch: F_i ~
    log-uniform(faces_range), n_prims ~ U{prims_range}, both from seed seed0 + i."""
    rng = np.random.default_rng(seed0 + i)
    nf = int(round(math.exp(rng.uniform(math.log(faces_range[0]), math.log(faces_range[1])))))
    npr = int(rng.integers(prims_range[0], prims_range[1] + 1))
    return nf, npr, max(20, min(200, nf // (2 * npr)))


def batch_mesh(i: int, seed0: int = 1000, faces_range=(5_000, 200_000), prims_range=(1, 50)) -> Mesh:
    """Mesh i of a batch: a wild union with the batch's face count and
    primitive count for i, generated with seed seed0 + i."""
    nf, npr, min_faces = batch_mesh_params(i, seed0, faces_range, prims_range)
    return wild_union(npr, nf, seed0 + i, min_faces=min_faces)


def batch_meshes(n: int = 512, seed0: int = 1000, faces_range=(5_000, 200_000),
                 prims_range=(1, 50)) -> list:
    """``n`` wild unions; mesh i has F_i ~ log-uniform(faces_range),
    n_prims ~ U{prims_range} and seed seed0 + i."""
    return [batch_mesh(i, seed0, faces_range, prims_range) for i in range(n)]
