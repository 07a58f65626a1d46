"""Seeded synthetic workloads shaped like the paper's experiments.

The paper (Sec. 6) solves the gravimetry Poisson problem on a regional box
(250 x 250 x 15) with measured densities that are not available here.  These
generators stand in for it with fixed-seed synthetic density anomalies on
axis-aligned tensor-product meshes:

* ``sphere_problem``   unit cube, 16^3 Q2 elements, 2x2x2 subdomains, one
                       sphere (R=0.2 at (0.5, 0.5, 0.6), 300 kg/m^3), p = 10.
* ``layered_problem``  unit cube, n^3 elements, three horizontal layers
                       (-200, 0, +250 kg/m^3 bottom to top) plus random
                       spheres (R ~ U[0.03, 0.1], drho ~ N(0, 150^2)).
* ``regional_problem`` 100 x 100 x 30 box, 128 x 128 x 48 elements graded
                       vertically (ratio 1.05, finest at the top surface),
                       8 x 8 x 3 uneven subdomains from jittered cut planes,
                       Gaussian random field (correlation length 5,
                       sigma = 100) plus a paraboloid basin of -250.
* ``slab_problem``     the paper's own set-up (Sec. 6): a 250 x 250 x 15 box
                       partitioned into slabs along x only (32, 64 or 128),
                       384 x 384 x 16 elements (19.5M Q2 nodes, near the
                       paper's 19.9M unknowns), layered crust with a buried
                       crater structure standing in for the measured model.

Everything here is input only: coordinates, per-element densities (x-fastest
flattening), element-index cut arrays, station coordinates and Robin
parameter samples.  No assembly or solver arithmetic lives here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

G_NEWTON = 6.672e-11  # m^3 kg^-1 s^-2, Sec. 2

__all__ = [
    "G_NEWTON", "Problem", "uniform_coords", "graded_coords", "equal_cuts",
    "jittered_cuts", "element_centroids", "sphere_density", "layered_density",
    "grf_basin_density", "sphere_problem", "layered_problem",
    "regional_problem", "batch_instances", "surface_stations", "crater_density", "slab_problem",
    "splitmix64", "log_uniform_p", "workload", "WORKLOADS",
]


@dataclass
class Problem:
    """One gravimetry problem: tensor mesh, density, decomposition, Robin p."""
    name: str
    xc: np.ndarray            # (nx+1,) element vertex x-coordinates
    yc: np.ndarray            # (ny+1,)
    zc: np.ndarray            # (nz+1,)
    drho: np.ndarray          # (nx*ny*nz,) kg/m^3, x-fastest
    cx: np.ndarray            # (sx+1,) element-index cuts in x
    cy: np.ndarray
    cz: np.ndarray
    p: float = 10.0           # Robin parameter (OO0, symmetric)
    inner_rtol: float = 1e-10  # subdomain PCG tolerance (Sec. 6: 1e-10)
    rtol: float = 1e-8        # Schwarz global relative residual
    meta: dict = field(default_factory=dict)

    @property
    def nx(self): return len(self.xc) - 1

    @property
    def ny(self): return len(self.yc) - 1

    @property
    def nz(self): return len(self.zc) - 1

    @property
    def n_nodes(self):
        return (2 * self.nx + 1) * (2 * self.ny + 1) * (2 * self.nz + 1)

    @property
    def n_dofs(self):
        """Interior (non-Dirichlet) Q2 nodes of the global problem."""
        return (2 * self.nx - 1) * (2 * self.ny - 1) * (2 * self.nz - 1)

    @property
    def n_sub(self):
        return (len(self.cx) - 1) * (len(self.cy) - 1) * (len(self.cz) - 1)


# ----------------------------------------------------------------- meshes --

def uniform_coords(n: int, length: float = 1.0) -> np.ndarray:
    return np.linspace(0.0, length, n + 1)


def graded_coords(n: int, length: float, ratio: float, fine_at_top: bool = True) -> np.ndarray:
    """Geometric grading: element sizes h0 * ratio^k summing to ``length``.

    With ``fine_at_top`` the smallest element touches z = length.
    """
    h0 = length * (ratio - 1.0) / (ratio ** n - 1.0)
    h = h0 * ratio ** np.arange(n)          # from the fine end outwards
    if fine_at_top:
        h = h[::-1]
    c = np.concatenate([[0.0], np.cumsum(h)])
    c[-1] = length
    return c


def equal_cuts(n_el: int, s: int) -> np.ndarray:
    if n_el % s:
        raise ValueError("equal cuts need n divisible by s")
    return np.arange(s + 1, dtype=np.int32) * (n_el // s)


def jittered_cuts(n_el: int, s: int, rng: np.random.Generator,
                  jitter: float = 0.3, min_el: int = 2) -> np.ndarray:
    """Cut planes at nominal i*n/s moved by U(-jitter, jitter) * spacing."""
    spacing = n_el / s
    cuts = [0]
    for i in range(1, s):
        c = int(round(i * spacing + rng.uniform(-jitter, jitter) * spacing))
        c = max(c, cuts[-1] + min_el)
        c = min(c, n_el - min_el * (s - i))
        cuts.append(c)
    cuts.append(n_el)
    return np.asarray(cuts, dtype=np.int32)


def element_centroids(xc, yc, zc):
    """Centroids as three (nz, ny, nx) arrays (x fastest when flattened)."""
    mx = 0.5 * (xc[:-1] + xc[1:])
    my = 0.5 * (yc[:-1] + yc[1:])
    mz = 0.5 * (zc[:-1] + zc[1:])
    Z, Y, X = np.meshgrid(mz, my, mx, indexing="ij")
    return X, Y, Z


# -------------------------------------------------------------- densities --

def sphere_density(xc, yc, zc, centre, radius, value):
    X, Y, Z = element_centroids(xc, yc, zc)
    r2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2
    return np.where(r2 <= radius * radius, float(value), 0.0).ravel()


def layered_density(xc, yc, zc, rng, n_spheres=20,
                    layers=(-200.0, 0.0, 250.0)):
    """Three equal-thickness z-layers (bottom to top) plus random spheres.

    Sphere centres ~ U[0.1, 0.9]^3 of the box, radii ~ U[0.03, 0.1] of the
    box's x-length, values ~ N(0, 150^2); overlapping contributions add.
    """
    X, Y, Z = element_centroids(xc, yc, zc)
    lx, ly, lz = xc[-1] - xc[0], yc[-1] - yc[0], zc[-1] - zc[0]
    rho = np.zeros_like(X)
    t = (Z - zc[0]) / lz
    rho += np.where(t < 1.0 / 3.0, layers[0], np.where(t < 2.0 / 3.0, layers[1], layers[2]))
    for _ in range(n_spheres):
        c = rng.uniform(0.1, 0.9, size=3) * np.array([lx, ly, lz]) + np.array([xc[0], yc[0], zc[0]])
        r = rng.uniform(0.03, 0.1) * lx
        v = rng.normal(0.0, 150.0)
        r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
        rho += np.where(r2 <= r * r, v, 0.0)
    return rho.ravel()


def _gauss_filter_axis(field, centres, ell, axis):
    d = centres[:, None] - centres[None, :]
    w = np.exp(-d * d / (2.0 * ell * ell))
    return np.moveaxis(np.tensordot(w, np.moveaxis(field, axis, 0), axes=(1, 0)), 0, axis)


def grf_basin_density(xc, yc, zc, rng, ell=5.0, sigma=100.0,
                      basin_centre=(50.0, 50.0), basin_radius=30.0,
                      basin_depth=6.0, basin_value=-250.0):
    """Gaussian random field plus a paraboloid low-density basin.

    White noise on the element-centroid grid is filtered by the separable
    Gaussian kernel exp(-r^2 / 2 ell^2) in physical coordinates, shifted to
    zero mean and scaled to standard deviation ``sigma`` exactly.  Elements
    whose centroid lies inside the bowl z > top - D (1 - r^2 / R^2), r < R,
    are overwritten with ``basin_value``.
    """
    X, Y, Z = element_centroids(xc, yc, zc)
    noise = rng.standard_normal(X.shape)
    mx = 0.5 * (xc[:-1] + xc[1:])
    my = 0.5 * (yc[:-1] + yc[1:])
    mz = 0.5 * (zc[:-1] + zc[1:])
    f = _gauss_filter_axis(noise, mz, ell, 0)
    f = _gauss_filter_axis(f, my, ell, 1)
    f = _gauss_filter_axis(f, mx, ell, 2)
    f = f - f.mean()
    f = f * (sigma / f.std())
    top = zc[-1]
    r2 = (X - basin_centre[0]) ** 2 + (Y - basin_centre[1]) ** 2
    bowl = (r2 < basin_radius ** 2) & (Z > top - basin_depth * (1.0 - r2 / basin_radius ** 2))
    f = np.where(bowl, basin_value, f)
    return f.ravel()


def crater_density(xc, yc, zc, rng, centre=(125.0, 125.0), rim_radius=100.0, cover=1.0,
                   lens_depth=3.0, lens_value=-250.0, uplift_radius=25.0, uplift_top=4.0,
                   uplift_bottom=11.0, uplift_value=200.0, ring=(35.0, 45.0), ring_value=100.0,
                   layers=(100.0, 0.0, -150.0), noise=10.0):
    """Layered crust with a buried impact structure, in km (top at zc[-1]).

    Layers (bottom third, middle third, top third): ``layers``.  Under a
    sediment cover of ``cover``: a low-density breccia lens filling the bowl
    top - cover - lens_depth (1 - r^2/R^2) < z < top - cover inside the rim
    radius R; a dense central uplift (r < uplift_radius, depths uplift_top to
    uplift_bottom below the surface); a peak ring (ring[0] < r < ring[1]) in
    the lens.  Plus white noise N(0, noise^2) per element.
    """
    X, Y, Z = element_centroids(xc, yc, zc)
    lz = zc[-1] - zc[0]
    t = (Z - zc[0]) / lz
    rho = np.where(t < 1.0 / 3.0, layers[0], np.where(t < 2.0 / 3.0, layers[1], layers[2]))
    top = zc[-1]
    r2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2
    depth = top - Z
    lens = (r2 < rim_radius ** 2) & (depth > cover) & \
           (depth < cover + lens_depth * (1.0 - r2 / rim_radius ** 2))
    rho = np.where(lens, lens_value, rho)
    ring_m = lens & (r2 > ring[0] ** 2) & (r2 < ring[1] ** 2)
    rho = np.where(ring_m, ring_value, rho)
    uplift = (r2 < uplift_radius ** 2) & (depth > uplift_top) & (depth < uplift_bottom)
    rho = np.where(uplift, uplift_value, rho)
    rho = rho + rng.normal(0.0, noise, size=rho.shape)
    return rho.ravel()


# ---------------------------------------------------------------- problems --

def sphere_problem(n: int = 16, s: int = 2, p: float = 10.0) -> Problem:
    xc = uniform_coords(n)
    drho = sphere_density(xc, xc, xc, (0.5, 0.5, 0.6), 0.2, 300.0)
    cuts = equal_cuts(n, s)
    return Problem(f"sphere_{n}^3_{s}^3", xc, xc.copy(), xc.copy(), drho,
                   cuts, cuts.copy(), cuts.copy(), p=p, inner_rtol=1e-12, rtol=1e-10)


def layered_problem(n: int = 64, s: int = 4, p: float = 10.0, seed: int = 0,
                    n_spheres: int = 20) -> Problem:
    rng = np.random.default_rng(seed)
    xc = uniform_coords(n)
    drho = layered_density(xc, xc, xc, rng, n_spheres=n_spheres)
    cuts = equal_cuts(n, s) if n % s == 0 else jittered_cuts(n, s, rng, 0.0)
    return Problem(f"layered_{n}^3_{s}^3", xc, xc.copy(), xc.copy(), drho,
                   cuts, cuts.copy(), cuts.copy(), p=p, rtol=1e-8)


def regional_problem(nx=128, ny=128, nz=48, sx=8, sy=8, sz=3, p=1.0, seed=0,
                     lx=100.0, ly=100.0, lz=30.0, grading=1.05) -> Problem:
    rng = np.random.default_rng(seed)
    xc = uniform_coords(nx, lx)
    yc = uniform_coords(ny, ly)
    zc = graded_coords(nz, lz, grading, fine_at_top=True)
    cx = jittered_cuts(nx, sx, rng)
    cy = jittered_cuts(ny, sy, rng)
    cz = jittered_cuts(nz, sz, rng)
    drho = grf_basin_density(xc, yc, zc, rng,
                             basin_centre=(0.5 * lx, 0.5 * ly))
    return Problem(f"regional_{nx}x{ny}x{nz}_{sx}x{sy}x{sz}", xc, yc, zc, drho,
                   cx, cy, cz, p=p, rtol=1e-8)


def slab_problem(nx=384, ny=384, nz=16, n_slabs=32, seed=0, lx=250.0, ly=250.0, lz=15.0,
                 p=1.0) -> Problem:
    """The paper's partition (Sec. 6): slabs along x only, one per subdomain,
    on a thin 250 x 250 x 15 box; stop test 1e-6 as in Table 2."""
    rng = np.random.default_rng(seed)
    xc = uniform_coords(nx, lx)
    yc = uniform_coords(ny, ly)
    zc = uniform_coords(nz, lz)
    drho = crater_density(xc, yc, zc, rng, centre=(0.5 * lx, 0.5 * ly), rim_radius=0.4 * lx)
    return Problem(f"slab_{nx}x{ny}x{nz}_{n_slabs}", xc, yc, zc, drho,
                   equal_cuts(nx, n_slabs), np.array([0, ny], dtype=np.int32),
                   np.array([0, nz], dtype=np.int32), p=p, rtol=1e-6)


def batch_instances(n_inst=64, lo=24, hi=40, seed=0, p_lo=2.0, p_hi=50.0):
    """Independent unit-cube problems with n ~ U{lo..hi}, 2x2x2 subdomains,
    their own layered density and their own log-uniform p."""
    rng = np.random.default_rng(seed)
    ps = log_uniform_p(seed + 1, n_inst, p_lo, p_hi)
    out = []
    for k in range(n_inst):
        n = int(rng.integers(lo, hi + 1))
        xc = uniform_coords(n)
        drho = layered_density(xc, xc, xc, rng)
        cuts = np.array([0, n // 2, n], dtype=np.int32)
        out.append(Problem(f"inst{k}_{n}^3", xc, xc.copy(), xc.copy(), drho,
                           cuts, cuts.copy(), cuts.copy(), p=float(ps[k]), rtol=1e-8))
    return out


def surface_stations(m=64, lx=1.0, ly=1.0, z=1.0):
    """m x m stations at cell centres of the top face, as (m*m, 3)."""
    t = (np.arange(m) + 0.5) / m
    Y, X = np.meshgrid(t * ly, t * lx, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(m * m, z)], axis=1)


# ---------------------------------------------------------- random p draws --

_MASK64 = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): n outputs as uint64."""
    out = np.empty(n, dtype=np.uint64)
    state = seed & _MASK64
    for i in range(n):
        state = (state + 0x9E3779B97F4A7C15) & _MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        out[i] = z ^ (z >> 31)
    return out


def log_uniform_p(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    """p = exp(log lo + u (log hi - log lo)), u = (x >> 11) * 2^-53."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))


# --------------------------------------------------------- named workloads --

def workload(name: str) -> Problem:
    """The named synthetic workloads used by tests and the benchmark."""
    if name == "sphere16":
        return sphere_problem(16, 2, 10.0)
    if name == "layered64":
        return layered_problem(64, 4, p=10.0, seed=0)
    if name == "layered48":
        return layered_problem(48, 3, p=10.0, seed=0)
    if name == "layered32":
        return layered_problem(32, 4, p=20.0, seed=0)
    if name == "regional":
        return regional_problem()
    if name == "regional_mid":
        # the regional workload's subdomain sizes and grading on a quarter of
        # its area and a third of its depth: 8 x 8 x 1 subdomains (profiling
        # captures that must stay at a few GB on the device)
        return regional_problem(nx=128, ny=128, nz=16, sx=8, sy=8, sz=1, p=1.6664, seed=0, lx=100.0, ly=100.0,
                                lz=10.0)
    if name == "layered160":
        return layered_problem(160, 8, p=10.0, seed=0)
    if name in ("slab32", "slab64", "slab128"):
        return slab_problem(n_slabs=int(name[4:]))
    raise KeyError(name)


WORKLOADS = ("sphere16", "layered32", "layered64", "layered48", "regional", "regional_mid", "layered160",
             "slab32", "slab64", "slab128")
