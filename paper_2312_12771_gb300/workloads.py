"""Seeded synthetic RVE workloads (microstructures, materials, macro loads).

This module only *generates inputs*: element phase arrays, per-RVE material
tables and macro deformation gradients.  It holds none of the method's
arithmetic (no kinematics, no element integrals, no solves), so both the CUDA
path and the FP64 oracle may consume what it produces.

Conventions shared by every consumer
------------------------------------
* An RVE is the unit cell [0,1]^d meshed by N^d equal elements (Q4 in 2D,
  Hex8 in 3D).  Element (ex, ey[, ez]) has flat index ex + N*ey (+ N*N*ez).
* ``phase`` is uint8 per element; phase 0 is the matrix, phase 1 the
  inclusion / fiber / second laminate layer.
* ``mat`` is float64 [nrve][nphase][4] = (model, p1, p2, p3):
  model 0 = linear isotropic elastic (p1=E, p2=nu),
  model 1 = compressible Neo-Hooke (p1=mu, p2=kappa).  p3 is unused (0).
* ``Fbar`` is float64 [nrve][d][d], row-major (F_iJ, J fastest).

Random numbers come from splitmix64 streams keyed by (seed, rve, stream) so
that any RVE of a batch can be regenerated alone.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GLOBAL_SEED = 2312_12771
MASK64 = (1 << 64) - 1

MODEL_LINEAR = 0
MODEL_NEOHOOKE = 1
MODEL_MOONEY_RIVLIN = 2


# --------------------------------------------------------------------------
# counter-based generator: splitmix64 (Steele, Lea & Flood 2014)
# --------------------------------------------------------------------------
def _splitmix64_next(state: int) -> tuple[int, int]:
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


class Stream:
    """A splitmix64 stream keyed by (seed, rve, stream id)."""

    def __init__(self, seed: int, rve: int, stream: int = 0):
        key = (seed * 0x100000001B3 + rve * 0x9E3779B1 + stream * 0x85EBCA77) & MASK64
        self.state = key
        # decorrelate neighbouring keys
        for _ in range(2):
            self.state, _ = _splitmix64_next(self.state)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        self.state, z = _splitmix64_next(self.state)
        return (z >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + int(self.uniform() * (hi - lo + 1))


# --------------------------------------------------------------------------
# microstructures (phase per element, decided at the element centroid)
# --------------------------------------------------------------------------
def _centroids(N: int, d: int) -> np.ndarray:
    c = (np.arange(N) + 0.5) / N
    grids = np.meshgrid(*([c] * d), indexing="ij")
    # flat index ex + N*ey (+N*N*ez): x must vary fastest -> reverse axes
    pts = np.stack([g.transpose(tuple(range(d))[::-1]).reshape(-1) for g in grids], axis=1)
    return pts  # [N^d][d], pts[e] = (x, y[, z]) of element e


def laminate_phase(N: int, rows_per_layer: int = 2) -> np.ndarray:
    """Layers along x: element row ey is phase 1 iff floor(ey/rows) is odd."""
    ey = np.repeat(np.arange(N), N)
    return ((ey // rows_per_layer) % 2).astype(np.uint8)


def _min_image(delta: np.ndarray) -> np.ndarray:
    return delta - np.round(delta)


def inclusion_phase(N: int, d: int, centres, radii) -> np.ndarray:
    """Phase 1 where the element centroid lies strictly inside any inclusion
    (minimum-image distance, so inclusions wrap periodically)."""
    pts = _centroids(N, d)
    ph = np.zeros(N ** d, dtype=np.uint8)
    for c, r in zip(centres, radii):
        dd = _min_image(pts - np.asarray(c, dtype=np.float64)[None, :])
        inside = np.einsum("ij,ij->i", dd, dd) < r * r
        ph[inside] = 1
    return ph


def fiber_phase(N: int, vf: float = 0.3) -> np.ndarray:
    """One centred circular fiber of volume fraction vf (2D)."""
    return inclusion_phase(N, 2, [(0.5, 0.5)], [math.sqrt(vf / math.pi)])


def sphere_phase(N: int, vf: float = 0.2) -> np.ndarray:
    """One centred spherical inclusion of volume fraction vf (3D)."""
    r = (3.0 * vf / (4.0 * math.pi)) ** (1.0 / 3.0)
    return inclusion_phase(N, 3, [(0.5, 0.5, 0.5)], [r])


def cross_phase(N: int, width: float = 1.0 / 3.0) -> np.ndarray:
    """Centred cross of the given width (fraction of the cell side) in phase 1,
    the rest phase 0 -- the membrane RVE of Section 5.2 ((-3,3)^2 mm with a
    2 mm cross: width 1/3), element phase by centroid."""
    pts = _centroids(N, 2)
    inside = (np.abs(pts[:, 0] - 0.5) < 0.5 * width) | (np.abs(pts[:, 1] - 0.5) < 0.5 * width)
    return inside.astype(np.uint8)


def random_inclusions(seed: int, rve: int, d: int = 2, nmin: int = 1, nmax: int = 6,
                      rmin: float = 0.05, rmax: float = 0.15, max_tries: int = 10000):
    """1..6 non-overlapping periodic circles: count U{nmin..nmax}, radius
    U[rmin,rmax], centre U[0,1)^d; rejection on minimum-image centre distance
    > r1 + r2."""
    s = Stream(seed, rve, 1)
    count = s.randint(nmin, nmax)
    centres, radii = [], []
    tries = 0
    while len(centres) < count and tries < max_tries:
        tries += 1
        r = rmin + (rmax - rmin) * s.uniform()
        c = np.array([s.uniform() for _ in range(d)])
        ok = True
        for c2, r2 in zip(centres, radii):
            dd = _min_image(c - c2)
            if math.sqrt(float(dd @ dd)) <= r + r2:
                ok = False
                break
        if ok:
            centres.append(c)
            radii.append(r)
    return centres, radii


# --------------------------------------------------------------------------
# material tables
# --------------------------------------------------------------------------
def linear_mat(E0: float, nu0: float, E1: float, nu1: float) -> np.ndarray:
    return np.array([[MODEL_LINEAR, E0, nu0, 0.0], [MODEL_LINEAR, E1, nu1, 0.0]])


def neohooke_mat(mu0: float, kappa0: float, mu1: float, kappa1: float) -> np.ndarray:
    return np.array([[MODEL_NEOHOOKE, mu0, kappa0, 0.0], [MODEL_NEOHOOKE, mu1, kappa1, 0.0]])


def mooney_rivlin_mat(p0, p1) -> np.ndarray:
    """Two Mooney-Rivlin phases, p = (alpha, beta, kappa)."""
    return np.array([[MODEL_MOONEY_RIVLIN, *p0], [MODEL_MOONEY_RIVLIN, *p1]], dtype=np.float64)


# the two membrane materials of Section 5.2: (alpha, beta, kappa)
MEMBRANE_MATERIAL_1 = (27.0, 18.0, 60.0)
MEMBRANE_MATERIAL_2 = (13.5, 6.5, 30.0)
MEMBRANE_TRACTION = (-5.0, 10.0)


def cook_mesh(nx: int, ny: int):
    """Cook's membrane of Section 5.2: the quadrilateral with corners (0,0),
    (480,440), (480,600), (0,440), meshed by nx x ny bilinear elements
    (straight lines between corresponding points of the bottom and top
    edges).  Node n = ix + (nx+1) iy, element nodes ordered
    (ix,iy), (ix+1,iy), (ix,iy+1), (ix+1,iy+1).  Returns X [nnode][2],
    conn [nelem][4], the left-edge nodes (clamped) and the right-edge nodes
    (loaded), bottom to top."""
    xs = np.linspace(0.0, 480.0, nx + 1)
    X = np.zeros(((nx + 1) * (ny + 1), 2))
    for iy in range(ny + 1):
        t = iy / ny
        for ix in range(nx + 1):
            x = xs[ix]
            lo, hi = 11.0 / 12.0 * x, x / 3.0 + 440.0
            X[ix + (nx + 1) * iy] = (x, lo + t * (hi - lo))
    conn = []
    for iy in range(ny):
        for ix in range(nx):
            n0 = ix + (nx + 1) * iy
            conn.append([n0, n0 + 1, n0 + nx + 1, n0 + nx + 2])
    left = np.array([(nx + 1) * iy for iy in range(ny + 1)])
    right = np.array([nx + (nx + 1) * iy for iy in range(ny + 1)])
    return X, np.array(conn, dtype=np.int32), left, right


# --------------------------------------------------------------------------
# batches
# --------------------------------------------------------------------------
@dataclass
class RveBatch:
    """A batch of RVEs of one mesh size per RVE (sizes may differ)."""
    d: int
    N: np.ndarray                 # int32 [nrve]
    phase: list                   # list of uint8 [N^d] arrays
    mat: np.ndarray               # float64 [nrve][nphase][4]
    Fbar: np.ndarray              # float64 [nrve][d][d]
    meta: dict = field(default_factory=dict)

    @property
    def nrve(self) -> int:
        return len(self.N)

    def phase_concat(self) -> np.ndarray:
        return np.concatenate(self.phase).astype(np.uint8)

    def subset(self, idx) -> "RveBatch":
        idx = list(idx)
        return RveBatch(self.d, self.N[idx].copy(), [self.phase[i] for i in idx],
                        self.mat[idx].copy(), self.Fbar[idx].copy(), dict(self.meta))


def laminate_batch(nrve: int = 64, N: int = 8, strain: float = 1e-3) -> RveBatch:
    """Two-phase laminate, E1=1 / E2=10, nu=0.3, uniaxial strain H=diag(strain,0)."""
    ph = laminate_phase(N)
    mat = np.repeat(linear_mat(1.0, 0.3, 10.0, 0.3)[None], nrve, axis=0)
    F = np.repeat((np.eye(2) + np.diag([strain, 0.0]))[None], nrve, axis=0)
    return RveBatch(2, np.full(nrve, N, np.int32), [ph] * nrve, mat, F,
                    {"workload": f"laminate {N}x{N} Q4, {nrve} RVEs"})


def cook_batch(nrve: int, N: int = 30) -> RveBatch:
    """Membrane RVEs of Section 5.2: the cross microstructure (phase 1 = the
    second material) at every macro Gauss point, Fbar = I."""
    ph = cross_phase(N)
    mat = np.broadcast_to(mooney_rivlin_mat(MEMBRANE_MATERIAL_1, MEMBRANE_MATERIAL_2), (nrve, 2, 4)).copy()
    F = np.broadcast_to(np.eye(2), (nrve, 2, 2)).copy()
    return RveBatch(2, np.full(nrve, N, np.int32), [ph] * nrve, mat, F,
                    meta={"kind": "cook membrane cross", "N": N})


def fiber_batch(nrve: int = 4096, N: int = 32, seed: int = GLOBAL_SEED, strain: float = 1e-3,
                dF_scale: float = 0.0) -> RveBatch:
    """Centred fiber vf=0.3, E_f=10, E_m=1(1+0.05u) u~U[-1,1] per RVE, nu=0.3."""
    ph = fiber_phase(N)
    mat = np.zeros((nrve, 2, 4))
    F = np.zeros((nrve, 2, 2))
    for r in range(nrve):
        s = Stream(seed, r, 0)
        Em = 1.0 * (1.0 + 0.05 * (2.0 * s.uniform() - 1.0))
        mat[r] = linear_mat(Em, 0.3, 10.0, 0.3)
        dF = np.array([[s.uniform(), s.uniform()], [s.uniform(), s.uniform()]]) * 2.0 - 1.0
        F[r] = np.eye(2) + np.diag([strain, 0.0]) + dF_scale * dF
    return RveBatch(2, np.full(nrve, N, np.int32), [ph] * nrve, mat, F,
                    {"workload": f"fiber vf=0.3 {N}x{N} Q4, {nrve} RVEs"})


def inclusion_batch(nrve: int, N, seed: int = GLOBAL_SEED, mu_m: float = 1.0,
                    ratio: float = 20.0, stretch: float = 1.0, d: int = 2) -> RveBatch:
    """Neo-Hooke RVEs with 1..6 random periodic inclusions, mu_i/mu_m=ratio,
    kappa=10 mu; N may be an int or an array of per-RVE sizes."""
    Ns = np.full(nrve, N, np.int32) if np.isscalar(N) else np.asarray(N, np.int32)
    phases = []
    for r in range(nrve):
        c, rad = random_inclusions(seed, r, d=d)
        phases.append(inclusion_phase(int(Ns[r]), d, c, rad))
    mat = np.repeat(neohooke_mat(mu_m, 10 * mu_m, ratio * mu_m, 10 * ratio * mu_m)[None], nrve, 0)
    F = np.repeat(np.diag([stretch] + [1.0] * (d - 1))[None], nrve, axis=0)
    return RveBatch(d, Ns, phases, mat, F, {"workload": f"NH inclusions, {nrve} RVEs"})


def sphere_batch(nrve: int, N: int = 8, gamma: float = 0.0, ratio: float = 10.0) -> RveBatch:
    """3D Neo-Hooke RVEs with a centred sphere vf=0.2, mu_i/mu_m=ratio, kappa=10 mu,
    simple shear F = I + gamma e1 x e2."""
    ph = sphere_phase(N)
    mat = np.repeat(neohooke_mat(1.0, 10.0, ratio, 10 * ratio)[None], nrve, 0)
    F0 = np.eye(3)
    F0[0, 1] = gamma
    F = np.repeat(F0[None], nrve, axis=0)
    return RveBatch(3, np.full(nrve, N, np.int32), [ph] * nrve, mat, F,
                    {"workload": f"sphere vf=0.2 {N}^3 Hex8, {nrve} RVEs"})


def serving_sizes(seed: int, nreq: int, sizes=(16, 24, 32, 48)) -> np.ndarray:
    """Per-request mesh size drawn uniformly from ``sizes``."""
    out = np.empty(nreq, np.int32)
    for r in range(nreq):
        out[r] = sizes[Stream(seed, r, 2).randint(0, len(sizes) - 1)]
    return out


def poisson_arrivals(seed: int, nreq: int, rate: float) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    s = Stream(seed, 0, 3)
    t, out = 0.0, np.empty(nreq)
    for r in range(nreq):
        t += -math.log(1.0 - s.uniform()) / rate
        out[r] = t
    return out


def perturbed_F(batch: RveBatch, seed: int, scale: float) -> np.ndarray:
    """Seeded perturbation of each RVE's Fbar (entries U[-scale, scale])."""
    out = batch.Fbar.copy()
    d = batch.d
    for r in range(batch.nrve):
        s = Stream(seed, r, 4)
        for i in range(d):
            for j in range(d):
                out[r, i, j] += scale * (2.0 * s.uniform() - 1.0)
    return out
