"""Seeded synthetic inputs: meshes, areas, normals, SH transfer, lights, materials.

This module generates the *inputs* of the translucent-transfer method and holds
none of its arithmetic (no dipole, PCA, transfer, wavelet or relight code).  It
is the only module shared by the FP64 oracle tests and the CUDA-path tests.

The paper's scenes (Angel, Beethoven, Candle; Section 5) are not available, so
icospheres stand in for them:

* Mesh.  The sphere is cut into the 10 rhombic charts of the icosahedron (five
  northern, five southern), each sampled by a nu x nu grid, plus the two poles:
  10*nu^2 + 2 vertices.  This plays the role of the paper's regular
  "M x 2^n x 2^n" wavelet domain (Section 3.1) with M = 10 charts.  Vertex id of
  chart d, row r, column c is d*nu^2 + r*nu + c; the poles are 10*nu^2 (north)
  and 10*nu^2 + 1 (south).  Each icosahedron face is subdivided uniformly and the
  points are projected onto the unit sphere.
* Displacement.  Radius 1 + amp * n(p) with n a seeded 3D lattice value noise
  (splitmix64 lattice values, quintic-fade trilinear interpolation, octave o at
  frequency 2*2^o with weight 0.5^o, normalised by the weight sum).
* Scale.  Every mesh is scaled by 20 mm.
* Area A_i.  Barycentric cell area: one third of the areas of the flat triangles
  incident to vertex i (mm^2).
* Transfer T[j, i].  Irradiance transfer of real orthonormal SH basis j at
  vertex i under the clamped cosine (Section 4, ambient light with V = 1):
  T[j, i] = Ahat_l * Y_j(n_i), Ahat = (pi, 2pi/3, pi/4, 0, -pi/24) for l = 0..4,
  j = l^2 + l + m.  Exact on convex meshes; on displaced meshes it is the
  unshadowed transfer with area-weighted vertex normals.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MESH_SCALE_MM = 20.0

# Marble (RGB) of the small configuration: sigma_a, sigma_s' in 1/mm, eta.
MARBLE_SIGMA_A = (0.0021, 0.0041, 0.0071)
MARBLE_SIGMA_S = (2.19, 2.62, 3.00)
MARBLE_ETA = 1.3

# Material ranges of the PCA sample (natural log, 1/mm).
LOG_SIGMA_A_RANGE = (-7.0, 0.0)
LOG_SIGMA_S_RANGE = (-1.0, 2.0)

# Clamped-cosine SH convolution coefficients Ahat_l, l = 0..4 (Funk-Hecke).
_AHAT = (math.pi, 2.0 * math.pi / 3.0, math.pi / 4.0, 0.0, -math.pi / 24.0)

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


# ----------------------------------------------------------------------------
# Icosahedral chart mesh
# ----------------------------------------------------------------------------
def _icosahedron() -> np.ndarray:
    """12 unit vertices: 0 north pole, 1..5 upper ring, 6..10 lower ring, 11 south."""
    lat = math.atan(0.5)
    v = [(0.0, 0.0, 1.0)]
    for k in range(5):
        lon = 2.0 * math.pi * k / 5.0
        v.append((math.cos(lat) * math.cos(lon), math.cos(lat) * math.sin(lon), math.sin(lat)))
    for k in range(5):
        lon = 2.0 * math.pi * k / 5.0 + math.pi / 5.0
        v.append((math.cos(lat) * math.cos(lon), math.cos(lat) * math.sin(lon), -math.sin(lat)))
    v.append((0.0, 0.0, -1.0))
    return np.asarray(v, dtype=np.float64)


def _diamond_corners(d: int) -> tuple[int, int, int, int]:
    """Corners (P00, P10, P01, P11) of chart d; the chart diagonal is P10-P01."""
    if d < 5:
        k = d
        return 0, 1 + k, 1 + (k + 1) % 5, 6 + k
    k = d - 5
    return 1 + (k + 1) % 5, 6 + k, 6 + (k + 1) % 5, 11


def _grid_keys(nu: int, d: int, r: np.ndarray, c: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Exact key of chart-d grid point (r, c) and its (unnormalised) flat position.

    A point of a subdivided icosahedron face is an integer barycentric
    combination (w0 V_a + w1 V_b + w2 V_c) / nu of three corners.  The sorted list
    of (corner, weight) pairs with nonzero weight identifies the point exactly,
    whichever chart computes it.
    """
    P00, P10, P01, P11 = _diamond_corners(d)
    lower = (r + c) <= nu
    vid = np.empty(r.shape + (3,), dtype=np.int64)
    w = np.empty(r.shape + (3,), dtype=np.int64)
    vid[..., 0] = np.where(lower, P00, P11)
    vid[..., 1] = np.where(lower, P10, P01)
    vid[..., 2] = np.where(lower, P01, P10)
    w[..., 0] = np.where(lower, nu - r - c, r + c - nu)
    w[..., 1] = np.where(lower, r, nu - r)
    w[..., 2] = np.where(lower, c, nu - c)
    ico = _icosahedron()
    pos = (w[..., :, None] * ico[vid]).sum(axis=-2) / float(nu)
    # canonical key
    vid_k = np.where(w > 0, vid, 99)
    order = np.argsort(vid_k, axis=-1, kind="stable")
    vs = np.take_along_axis(vid_k, order, axis=-1)
    ws = np.take_along_axis(w, order, axis=-1)
    code = np.where(vs == 99, 0, vs * (nu + 1) + ws + 1)
    base = 12 * (nu + 1) + 1
    key = code[..., 0] * base * base + code[..., 1] * base + code[..., 2]
    return key, pos


@dataclass
class Mesh:
    """A chart-ordered icosphere mesh (positions in mm)."""
    nu: int
    pos: np.ndarray        # (N, 3) float64, mm
    tris: np.ndarray       # (F, 3) int64, outward winding
    area: np.ndarray       # (N,) float64, barycentric cell area, mm^2
    normal: np.ndarray     # (N, 3) float64, unit area-weighted vertex normals

    @property
    def n(self) -> int:
        return self.pos.shape[0]


def icosphere_unit(nu: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit-sphere vertices (N,3) and triangles (F,3) of the 10-chart icosphere."""
    if nu < 1:
        raise ValueError("nu must be >= 1")
    n = 10 * nu * nu + 2
    # owned points: rows r in [1, nu], cols c in [0, nu-1] of each chart
    rr, cc = np.meshgrid(np.arange(1, nu + 1), np.arange(0, nu), indexing="ij")
    keys = np.empty(n, dtype=np.int64)
    flat = np.empty((n, 3), dtype=np.float64)
    for d in range(10):
        k, p = _grid_keys(nu, d, rr, cc)
        keys[d * nu * nu:(d + 1) * nu * nu] = k.reshape(-1)
        flat[d * nu * nu:(d + 1) * nu * nu] = p.reshape(-1, 3)
    base = 12 * (nu + 1) + 1
    keys[n - 2] = (0 * (nu + 1) + nu + 1) * base * base   # north pole: corner 0, weight nu
    keys[n - 1] = (11 * (nu + 1) + nu + 1) * base * base  # south pole: corner 11, weight nu
    flat[n - 2] = (0.0, 0.0, 1.0)
    flat[n - 1] = (0.0, 0.0, -1.0)
    order = np.argsort(keys)
    sorted_keys = keys[order]
    if np.any(np.diff(sorted_keys) == 0):
        raise RuntimeError("duplicate vertex keys")
    pos = flat / np.linalg.norm(flat, axis=1, keepdims=True)

    # triangles: every chart's (nu x nu) quads split along the chart diagonal direction
    gr, gc = np.meshgrid(np.arange(nu + 1), np.arange(nu + 1), indexing="ij")
    tris = []
    for d in range(10):
        k, _ = _grid_keys(nu, d, gr, gc)
        loc = np.searchsorted(sorted_keys, k)
        if np.any(sorted_keys[np.minimum(loc, n - 1)] != k):
            raise RuntimeError("grid point without an owner")
        gid = order[loc]
        a = gid[:-1, :-1]
        b = gid[1:, :-1]
        c = gid[:-1, 1:]
        e = gid[1:, 1:]
        tris.append(np.stack([a, b, c], axis=-1).reshape(-1, 3))
        tris.append(np.stack([e, c, b], axis=-1).reshape(-1, 3))
    tris = np.concatenate(tris, axis=0)
    return pos, tris


def _splitmix64(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _MASK64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
        return z ^ (z >> np.uint64(31))


def _lattice(seed: int, octave: int, ix: np.ndarray, iy: np.ndarray, iz: np.ndarray) -> np.ndarray:
    """Lattice value in [-1, 1) from splitmix64 chained over (seed, octave, ix, iy, iz)."""
    h = _splitmix64(np.full(ix.shape, np.uint64(seed & 0xFFFFFFFFFFFFFFFF)))
    for v in (np.full(ix.shape, octave, dtype=np.int64), ix, iy, iz):
        h = _splitmix64(h ^ v.astype(np.int64).view(np.uint64))
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


def value_noise(p: np.ndarray, seed: int, octaves: int) -> np.ndarray:
    """Seeded multi-octave 3D lattice value noise at points p (N,3); range [-1, 1]."""
    total = np.zeros(p.shape[0], dtype=np.float64)
    wsum = 0.0
    for o in range(octaves):
        freq = 2.0 * (2.0 ** o)
        wgt = 0.5 ** o
        q = p * freq
        i0 = np.floor(q).astype(np.int64)
        t = q - i0
        f = t * t * t * (t * (t * 6.0 - 15.0) + 10.0)
        acc = np.zeros(p.shape[0], dtype=np.float64)
        for dx in (0, 1):
            wx = f[:, 0] if dx else 1.0 - f[:, 0]
            for dy in (0, 1):
                wy = f[:, 1] if dy else 1.0 - f[:, 1]
                for dz in (0, 1):
                    wz = f[:, 2] if dz else 1.0 - f[:, 2]
                    acc += wx * wy * wz * _lattice(seed, o, i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz)
        total += wgt * acc
        wsum += wgt
    return total / wsum


def mesh_from_unit(nu: int, unit: np.ndarray, tris: np.ndarray, radius: np.ndarray) -> Mesh:
    pos = unit * radius[:, None] * MESH_SCALE_MM
    e1 = pos[tris[:, 1]] - pos[tris[:, 0]]
    e2 = pos[tris[:, 2]] - pos[tris[:, 0]]
    cr = np.cross(e1, e2)
    tri_area = 0.5 * np.linalg.norm(cr, axis=1)
    area = np.zeros(pos.shape[0])
    nrm = np.zeros_like(pos)
    for a in range(3):
        np.add.at(area, tris[:, a], tri_area / 3.0)
        np.add.at(nrm, tris[:, a], cr)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return Mesh(nu=nu, pos=pos, tris=tris, area=area, normal=nrm)


def icosphere(nu: int, amp: float = 0.0, octaves: int = 3, seed: int = 0) -> Mesh:
    """Chart-ordered icosphere of 10*nu^2+2 vertices, radius 20 mm, optionally displaced."""
    unit, tris = icosphere_unit(nu)
    if amp != 0.0:
        radius = 1.0 + amp * value_noise(unit, seed, octaves)
    else:
        radius = np.ones(unit.shape[0])
    return mesh_from_unit(nu, unit, tris, radius)


# ----------------------------------------------------------------------------
# Real spherical harmonics and the SH irradiance transfer
# ----------------------------------------------------------------------------
def sh_real(order: int, dirs: np.ndarray) -> np.ndarray:
    """Real orthonormal SH Y_j(dirs), j = l^2 + l + m, l < order.  Returns (order^2, N)."""
    x, y, z = dirs[:, 0], dirs[:, 1], np.clip(dirs[:, 2], -1.0, 1.0)
    n = dirs.shape[0]
    phi = np.arctan2(y, x)
    st = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    # associated Legendre P_l^m(z) without the Condon-Shortley phase
    P = {}
    P[(0, 0)] = np.ones(n)
    for m in range(1, order):
        P[(m, m)] = P[(m - 1, m - 1)] * (2 * m - 1) * st
    for m in range(0, order):
        if m + 1 < order:
            P[(m + 1, m)] = z * (2 * m + 1) * P[(m, m)]
        for l in range(m + 2, order):
            P[(l, m)] = ((2 * l - 1) * z * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    Y = np.empty((order * order, n))
    for l in range(order):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                v = K * P[(l, 0)]
            elif m > 0:
                v = math.sqrt(2.0) * K * np.cos(m * phi) * P[(l, am)]
            else:
                v = math.sqrt(2.0) * K * np.sin(am * phi) * P[(l, am)]
            Y[l * l + l + m] = v
    return Y


def sh_transfer(normals: np.ndarray, J: int) -> np.ndarray:
    """T[j, i] = Ahat_l Y_j(n_i): clamped-cosine irradiance transfer, (J, N) float64."""
    order = int(round(math.sqrt(J)))
    if order * order != J or order > len(_AHAT):
        raise ValueError("J must be a square <= 25")
    Y = sh_real(order, normals)
    for l in range(order):
        Y[l * l:(l + 1) * (l + 1)] *= _AHAT[l]
    return Y


def sh_light(J: int, seed: int = 0) -> np.ndarray:
    """Random SH light coefficients l_j ~ N(0, 1)."""
    return np.random.default_rng(seed).standard_normal(J)


# ----------------------------------------------------------------------------
# Materials
# ----------------------------------------------------------------------------
def pca_materials(n: int = 256, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """PCA sample materials: ln sigma_a ~ U[-7,0] (drawn first), ln sigma_s' ~ U[-1,2]."""
    rng = np.random.default_rng(seed)
    sa = np.exp(rng.uniform(*LOG_SIGMA_A_RANGE, size=n))
    ss = np.exp(rng.uniform(*LOG_SIGMA_S_RANGE, size=n))
    return sa, ss


def edit_materials(n: int, seed: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Random RGB material edits: sigma_a, sigma_s' (n,3) log-uniform in the PCA ranges, eta ~ U[1.2,1.5]."""
    rng = np.random.default_rng(seed)
    sa = np.exp(rng.uniform(*LOG_SIGMA_A_RANGE, size=(n, 3)))
    ss = np.exp(rng.uniform(*LOG_SIGMA_S_RANGE, size=(n, 3)))
    eta = rng.uniform(1.2, 1.5, size=n)
    return sa, ss, eta


def marble(n: int = 1) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    sa = np.tile(np.asarray(MARBLE_SIGMA_A, dtype=np.float64), (n, 1))
    ss = np.tile(np.asarray(MARBLE_SIGMA_S, dtype=np.float64), (n, 1))
    return sa, ss, np.full(n, MARBLE_ETA)


def sample_rows(n: int, count: int, seed: int = 7) -> np.ndarray:
    """Sorted sample of output vertices (uniform without replacement)."""
    count = min(count, n)
    return np.sort(np.random.default_rng(seed).choice(n, size=count, replace=False))


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------
@dataclass
class Scene:
    mesh: Mesh
    K: int
    J: int
    T: np.ndarray      # (J, N) float64
    light: np.ndarray  # (J,) float64

    @property
    def n(self) -> int:
        return self.mesh.n


def make_scene(nu: int, K: int, J: int, amp: float = 0.0, octaves: int = 3,
               seed: int = 0, light_seed: int = 0) -> Scene:
    mesh = icosphere(nu, amp, octaves, seed)
    return Scene(mesh=mesh, K=K, J=J, T=sh_transfer(mesh.normal, J), light=sh_light(J, light_seed))


# The five workloads: (nu, K, J, amp, octaves, noise seed)
WORKLOADS = {
    "sphere2562_k8_j9": dict(nu=16, K=8, J=9, amp=0.0, octaves=3, seed=0),
    "disp40962_k12_j16": dict(nu=64, K=12, J=16, amp=0.1, octaves=3, seed=1),
    "disp163842_k16_j25": dict(nu=128, K=16, J=25, amp=0.15, octaves=5, seed=2),
}


def batched_nus(n_mesh: int = 256, seed: int = 4, nmin: int = 642, nmax: int = 40962) -> np.ndarray:
    """Chart sizes of the uneven batch: N* log-uniform on [nmin, nmax], nu = clamp(round(sqrt((N*-2)/10)), 8, 64)."""
    rng = np.random.default_rng(seed)
    nstar = np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=n_mesh))
    nu = np.rint(np.sqrt((nstar - 2.0) / 10.0)).astype(np.int64)
    return np.clip(nu, 8, 64)
