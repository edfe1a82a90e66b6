"""Seeded synthetic inputs for the transport library and its CPU oracle.

This module only builds inputs (density grids, optical properties, sources,
instruments and run settings).  It holds none of the transport arithmetic and
imports neither the CUDA binding nor the oracle, so both can be fed the same
arrays.  Every generator is deterministic for a given seed
(``numpy.random.default_rng``).

Workloads (shapes and value ranges follow the spiral-galaxy example of the
SKIRT paper, Sect. 2.5 and its ski file, and the component table, Table 1):

* ``uniform_cube``: uniform dust cube, central isotropic point source, one
  face-on frame (the plain-method case).
* ``disk_galaxy``: double-exponential stellar disk inside a double-exponential
  dust disk on a cartesian grid, several wavelengths with smooth synthetic
  optical properties, three frames at inclinations 0, 60 and 90 degrees.
* ``clumpy_octree``: Gaussian dust clumps binned onto an adaptive octree
  (Sect. 2.4), Plummer bulge plus exponential disk.
* ``lognormal_cube``: log-normal density field for gradient checks.
* ``batch_models``: many small independent models for the batched launcher.
* ``spiral_example``: the paper's worked spiral-galaxy example (Sect. 2.5)
  on a 3D power-law (PowCub) or equal-cell grid.
* ``clumpy_bintree``: the clumpy medium on a k-d tree (Table 1(d): BinTree).
* ``voronoi_disk``: the disk galaxy's dust on a Voronoi grid whose sites
  follow the dust density (Table 1(d): VoronoiDustGrid; Sect. 2.4).
* ``panchromatic_disk``: a stellar spectrum and dust that re-emits what it
  absorbs at its equilibrium temperature (Sect. 2.2, panchromatic mode).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np


@dataclass
class Grid:
    """Dust grid.  ``kind`` is ``"cartesian"`` (density float32 [nz, ny, nx],
    x fastest), ``"rectilinear"`` (the same with cell edges per axis in
    ``edges``: three float64 arrays of n + 1 increasing values),
    ``"octree"`` (``child`` int32 per node: index of the first of eight
    children, or -(leaf + 1) for a leaf; density float32 per leaf) or
    ``"bintree"`` (a k-d tree: ``child`` as for octrees but with two
    children, lower then upper half of the node's box split at its midpoint
    along ``split_axis`` int8 per node) or ``"voronoi"`` (cell c holds the
    points of the domain nearest to ``sites[c]``; ``child`` int32 lists the
    neighbours of every cell, cell c's in ``child[offsets[c]:offsets[c+1]]``;
    density float32 per cell)."""
    kind: str
    bounds: np.ndarray  # float64 [xmin, xmax, ymin, ymax, zmin, zmax]
    density: np.ndarray
    child: Optional[np.ndarray] = None
    edges: Optional[list] = None
    split_axis: Optional[np.ndarray] = None  # k-d tree ("bintree"): split axis per node
    sites: Optional[np.ndarray] = None  # Voronoi: float64 [n, 3] generating sites
    offsets: Optional[np.ndarray] = None  # Voronoi: int64 [n + 1], neighbours of c in child[offsets[c]:offsets[c+1]]

    @property
    def n_cells(self) -> int:
        return int(self.density.size)

    @property
    def shape(self):
        """(nx, ny, nz) for cartesian grids."""
        nz, ny, nx = self.density.shape
        return nx, ny, nz


@dataclass
class Source:
    """Emission component: ``point`` (center), ``expdisk`` (center, scale_r =
    hR, scale_z = hz, disk in the xy plane) or ``plummer`` (center, scale_r =
    a).  ``lum``: luminosity per wavelength."""
    kind: str
    center: tuple
    lum: np.ndarray
    scale_r: float = 0.0
    scale_z: float = 0.0


@dataclass
class Instrument:
    """Frame instrument with parallel projection.  Angles in radians;
    ``half_x``/``half_y`` are half-widths of the field; ``channels`` is 1
    (total) or 3 (total, direct, scattered).  ``sed``: an SED instrument
    (one bin per wavelength: the flux received from the viewing direction,
    wherever it comes from; nx = ny = 1, the field is not used)."""
    inclination: float
    azimuth: float
    position_angle: float
    nx: int
    ny: int
    half_x: float
    half_y: float
    center_x: float = 0.0
    center_y: float = 0.0
    bilinear: bool = False
    channels: int = 1
    sed: bool = False


@dataclass
class Run:
    """Run settings: total packets per wavelength and termination rule."""
    n_per_lambda: int
    seed: int = 0
    w_min: float = 1e-4
    max_events: int = 1000
    weight_cut: bool = True


@dataclass
class Problem:
    name: str
    grid: Grid
    wavelengths: np.ndarray
    kappa: np.ndarray
    albedo: np.ndarray
    g: np.ndarray
    sources: List[Source]
    instruments: List[Instrument]
    run: Run
    meta: dict = field(default_factory=dict)
    # panchromatic mode: thermal emission of the dust cells [n_lambda, n_cells],
    # emitted instead of the sources (None: the sources emit)
    dust_lum: Optional[np.ndarray] = None

    @property
    def n_lambda(self) -> int:
        return int(len(self.kappa))


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def cartesian_grid(bounds, density) -> Grid:
    return Grid("cartesian", _f64(bounds), np.ascontiguousarray(density, dtype=np.float32))


def rectilinear_grid(edges, density) -> Grid:
    """Grid of cuboidal cells between the given edges (x, y, z)."""
    e = [np.ascontiguousarray(a, dtype=np.float64) for a in edges]
    bounds = [e[0][0], e[0][-1], e[1][0], e[1][-1], e[2][0], e[2][-1]]
    return Grid("rectilinear", _f64(bounds), np.ascontiguousarray(density, dtype=np.float32), edges=e)


def powcub_edges(lo, hi, n, ratio):
    """Cell edges of ``n`` cells on [lo, hi], symmetric about the centre, with
    widths growing by a constant factor from the centre outwards so that the
    outermost cell is ``ratio`` times as wide as the innermost (the power-law
    spacing of the PowCub grid, Table 1(d); ratio 1 gives equal cells).  An
    odd ``n`` has one central cell."""
    half = n // 2
    centre = 0.5 * (lo + hi)
    length = hi - lo
    if n % 2 == 0:
        steps = half - 1
        q = ratio ** (1.0 / steps) if steps > 0 else 1.0
        w = q ** np.arange(half)
        t = np.concatenate([[0.0], np.cumsum(w)])
        t *= 0.5 * length / t[-1]
        edges = np.concatenate([centre - t[::-1], centre + t[1:]])
    else:
        q = ratio ** (1.0 / half) if half > 0 else 1.0
        w = q ** np.arange(half + 1)  # w[0]: the central cell
        t = np.concatenate([[0.5 * w[0]], 0.5 * w[0] + np.cumsum(w[1:])])
        t *= 0.5 * length / t[-1]
        edges = np.concatenate([centre - t[::-1], centre + t])
    edges[0], edges[-1] = lo, hi
    return edges


def cell_centres_of(grid):
    """Cell-centre coordinates (x [nx], y [ny], z [nz]) of a cartesian or
    rectilinear grid."""
    if grid.kind == "rectilinear":
        return tuple(0.5 * (e[1:] + e[:-1]) for e in grid.edges)
    return cell_centres(grid.bounds, grid.shape)


def cell_centres(bounds, shape):
    """Cell-centre coordinates (x [nx], y [ny], z [nz]) of a cartesian grid."""
    nx, ny, nz = shape
    b = np.asarray(bounds, dtype=np.float64)
    xs = b[0] + (np.arange(nx) + 0.5) * (b[1] - b[0]) / nx
    ys = b[2] + (np.arange(ny) + 0.5) * (b[3] - b[2]) / ny
    zs = b[4] + (np.arange(nz) + 0.5) * (b[5] - b[4]) / nz
    return xs, ys, zs


def synthetic_optics(wavelengths_um, kappa_v):
    """Smooth synthetic dust optics with x = ln(lambda / 0.55 um):
    kappa = kappa_V exp(-1.3 x), albedo = clip(0.6 - 0.1 x^2, 0.3, 0.8),
    g = clip(0.6 - 0.15 x, 0, 0.9)."""
    x = np.log(np.asarray(wavelengths_um, dtype=np.float64) / 0.55)
    kappa = kappa_v * np.exp(-1.3 * x)
    albedo = np.clip(0.6 - 0.1 * x * x, 0.3, 0.8)
    g = np.clip(0.6 - 0.15 * x, 0.0, 0.9)
    return kappa, albedo, g


def sed_instrument(inclination_deg, azimuth=-math.pi / 2, channels=3) -> Instrument:
    """SED instrument viewing from inclination ``inclination_deg`` degrees."""
    return Instrument(math.radians(inclination_deg), azimuth, 0.0, 1, 1, 1.0, 1.0, channels=channels, sed=True)


def face_on(n, half, bilinear=False, channels=1) -> Instrument:
    """Frame looking down the +z axis; image x = model x, image y = model y."""
    return Instrument(0.0, -math.pi / 2, 0.0, n, n, half, half, bilinear=bilinear, channels=channels)


# ---------------------------------------------------------------- workloads
def uniform_cube(n_cells=32, half=1.0, axis_tau=1.0, albedo=0.6, g=0.5, n_pix=64,
                 n_packets=100_000, channels=1, source_pos=(0.0, 0.0, 0.0), rho=1.0) -> Problem:
    """Uniform cube [-half, half]^3 with ``n_cells``^3 cells.  ``axis_tau`` is
    the optical depth along the full x axis through the centre, so
    kappa rho = axis_tau / (2 half).  Central isotropic point source of unit
    luminosity; one face-on frame covering the cube."""
    b = [-half, half] * 3
    dens = np.full((n_cells,) * 3, rho, dtype=np.float32)
    kappa = axis_tau / (2.0 * half) / rho if rho > 0 else 1.0
    return Problem(
        name=f"uniform_cube_{n_cells}",
        grid=cartesian_grid(b, dens),
        wavelengths=_f64([0.55]),
        kappa=_f64([kappa]), albedo=_f64([albedo]), g=_f64([g]),
        sources=[Source("point", tuple(float(c) for c in source_pos), _f64([1.0]))],
        instruments=[face_on(n_pix, half, channels=channels)],
        run=Run(n_per_lambda=n_packets),
    )


def disk_galaxy(n_cells=256, n_lambda=10, n_pix=512, n_packets_total=100_000_000,
                face_on_tau_v=0.5, channels=1) -> Problem:
    """Edge-on disk galaxy.  Domain x, y in [-25, 25] kpc, z in [-3, 3] kpc.
    Dust rho = exp(-R/6 - |z|/0.2) sampled at cell centres, kappa_V chosen so
    that the face-on V-band optical depth through the centre is
    kappa_V * rho0 * 2 hz = ``face_on_tau_v``.  Stars: exponential disk
    hR = 4 kpc, hz = 0.35 kpc, unit luminosity per wavelength.  Wavelengths
    log-spaced 0.15 - 2.2 um.  Three ``n_pix``^2 frames at inclinations 0, 60
    and 90 degrees (azimuth -90 degrees), half-width 25 kpc.  The total packet
    count is split equally over the wavelengths."""
    bounds = [-25.0, 25.0, -25.0, 25.0, -3.0, 3.0]
    xs, ys, zs = cell_centres(bounds, (n_cells, n_cells, n_cells))
    R = np.sqrt(xs[None, None, :] ** 2 + ys[None, :, None] ** 2)
    dens = np.exp(-R / 6.0 - np.abs(zs)[:, None, None] / 0.2).astype(np.float32)
    wl = np.geomspace(0.15, 2.2, n_lambda)
    kappa, albedo, g = synthetic_optics(wl, face_on_tau_v / (2.0 * 0.2))
    instr = [Instrument(math.radians(inc), -math.pi / 2, 0.0, n_pix, n_pix, 25.0, 25.0, channels=channels)
             for inc in (0.0, 60.0, 90.0)]
    return Problem(
        name=f"disk_galaxy_{n_cells}",
        grid=cartesian_grid(bounds, dens),
        wavelengths=wl, kappa=kappa, albedo=albedo, g=g,
        sources=[Source("expdisk", (0.0, 0.0, 0.0), np.ones(n_lambda), scale_r=4.0, scale_z=0.35)],
        instruments=instr,
        run=Run(n_per_lambda=max(1, n_packets_total // n_lambda)),
    )


# Units of the spiral-galaxy example: lengths in pc, luminosity and dust mass
# in solar units.  Extinction per unit dust mass at 0.55 um: a synthetic
# Milky-Way-like 2.6e4 cm^2 / g (the paper's Draine & Li tables are not
# available), converted to pc^2 / Msun.
PC_CM = 3.0857e18
MSUN_G = 1.98892e33
KAPPA_V_CM2_G = 2.6e4
KAPPA_V_PC2_MSUN = KAPPA_V_CM2_G * MSUN_G / PC_CM ** 2


def _exp_disk_cell_means(edges, h_r, h_z, n_gauss=4, chunk=1 << 20):
    """Mean of exp(-R/h_r - |z|/h_z) over each cell of a rectilinear grid:
    an n_gauss^3-point Gauss-Legendre rule per cell (the paper's example
    averages random density samples per cell; a fixed rule keeps the input
    deterministic).  Returns float64 [nz, ny, nx]."""
    gx, gw = np.polynomial.legendre.leggauss(n_gauss)
    ex, ey, ez = (np.asarray(e, dtype=np.float64) for e in edges)
    nx, ny, nz = len(ex) - 1, len(ey) - 1, len(ez) - 1
    # z factor separates: mean of exp(-|z|/h_z) per z cell by the rule
    zc, zh = 0.5 * (ez[1:] + ez[:-1]), 0.5 * (ez[1:] - ez[:-1])
    fz = (np.exp(-np.abs(zc[:, None] + zh[:, None] * gx[None, :]) / h_z) * gw[None, :]).sum(axis=1) / 2.0
    xc, xh = 0.5 * (ex[1:] + ex[:-1]), 0.5 * (ex[1:] - ex[:-1])
    yc, yh = 0.5 * (ey[1:] + ey[:-1]), 0.5 * (ey[1:] - ey[:-1])
    xs = (xc[:, None] + xh[:, None] * gx[None, :])  # [nx, g]
    ys = (yc[:, None] + yh[:, None] * gx[None, :])  # [ny, g]
    w2 = (gw[:, None] * gw[None, :]) / 4.0          # [g, g]
    fxy = np.empty((ny, nx))
    for j0 in range(0, ny, max(1, chunk // (nx * n_gauss * n_gauss))):
        j1 = min(ny, j0 + max(1, chunk // (nx * n_gauss * n_gauss)))
        R = np.sqrt(ys[j0:j1, None, :, None] ** 2 + xs[None, :, None, :] ** 2)  # [j, nx, g, g]
        fxy[j0:j1] = (np.exp(-R / h_r) * w2[None, None]).sum(axis=(2, 3))
    return fz[:, None, None] * fxy[None, :, :]


def spiral_example(grid="powcub", n_xy=256, n_z=128, xy_ratio=20.0, z_ratio=50.0, n_packets=10_000_000,
                   n_pix=(1200, 300)) -> Problem:
    """The simple spiral galaxy of the paper's worked example (Sect. 2.5, its
    ski file): a stellar exponential disk (scale length 4400 pc, height
    500 pc, 1e11 Lsun at 0.55 um) and a dust exponential disk (6600 pc,
    250 pc, 4e7 Msun of dust), 1e7 packets at one wavelength, one frame
    "xz" at inclination 90 deg, azimuth -90 deg, 1200 x 300 pixels with
    extents 28000 x 7000 pc (taken as half-widths).  The paper's grid is 2D
    axisymmetric (logarithmic radially from 250 to 25000 pc, power-law
    vertically up to 7000 pc with ratio 50); here the same domain
    [-25000, 25000]^2 x [-7000, 7000] pc is a 3D grid: ``grid="powcub"``
    with power-law spaced edges (``xy_ratio`` horizontally, ``z_ratio``
    vertically) or ``grid="cartesian"`` with equal cells.  Cell densities are
    cell means (Gauss-Legendre rule).  Optics at 0.55 um: the synthetic
    kappa of KAPPA_V_PC2_MSUN, albedo 0.6, g 0.6."""
    h_r, h_z, mass = 6600.0, 250.0, 4e7
    rho0 = mass / (4.0 * math.pi * h_r * h_r * h_z)
    if grid == "powcub":
        edges = [powcub_edges(-25000.0, 25000.0, n_xy, xy_ratio), powcub_edges(-25000.0, 25000.0, n_xy, xy_ratio),
                 powcub_edges(-7000.0, 7000.0, n_z, z_ratio)]
    elif grid == "cartesian":
        edges = [-25000.0 + np.arange(n_xy + 1) * (50000.0 / n_xy), -25000.0 + np.arange(n_xy + 1) * (50000.0 / n_xy),
                 -7000.0 + np.arange(n_z + 1) * (14000.0 / n_z)]
        for e, hi in zip(edges, (25000.0, 25000.0, 7000.0)):
            e[-1] = hi
    else:
        raise ValueError(grid)
    dens = (rho0 * _exp_disk_cell_means(edges, h_r, h_z)).astype(np.float32)
    g = rectilinear_grid(edges, dens) if grid == "powcub" else cartesian_grid([-25000.0, 25000.0, -25000.0, 25000.0,
                                                                                -7000.0, 7000.0], dens)
    kappa, albedo, gg = synthetic_optics([0.55], KAPPA_V_PC2_MSUN)
    frame = Instrument(math.radians(90.0), math.radians(-90.0), 0.0, n_pix[0], n_pix[1], 28000.0, 7000.0)
    return Problem(
        name=f"spiral_example_{grid}",
        grid=g, wavelengths=_f64([0.55]), kappa=kappa, albedo=albedo, g=gg,
        sources=[Source("expdisk", (0.0, 0.0, 0.0), _f64([1e11]), scale_r=4400.0, scale_z=500.0)],
        instruments=[frame],
        run=Run(n_per_lambda=int(n_packets)),
        meta={"dust_mass": mass, "rho0": rho0, "kappa_v_pc2_msun": float(KAPPA_V_PC2_MSUN),
              "face_on_tau_v": float(KAPPA_V_PC2_MSUN * mass / (2.0 * math.pi * h_r * h_r)),
              "edge_on_tau_v": float(KAPPA_V_PC2_MSUN * mass / (2.0 * math.pi * h_r * h_z))},
    )


def panchromatic_optics(wavelengths_um, kappa_v):
    """Synthetic optics over a UV-to-submillimetre grid, x = ln(lambda / 0.55
    um): kappa = kappa_V exp(-1.3 x), albedo = clip(0.6 - 0.1 x^2, 0, 0.8)
    (no scattering far in the infrared), g = clip(0.6 - 0.15 x, 0, 0.9)."""
    x = np.log(np.asarray(wavelengths_um, dtype=np.float64) / 0.55)
    return kappa_v * np.exp(-1.3 * x), np.clip(0.6 - 0.1 * x * x, 0.0, 0.8), np.clip(0.6 - 0.15 * x, 0.0, 0.9)


def stellar_spectrum(wavelengths_um, t_star=5800.0, total=1.0):
    """Luminosity per wavelength bin of a blackbody star of temperature
    t_star (bins centred on the wavelengths on a logarithmic scale), scaled
    to `total`."""
    lam = np.asarray(wavelengths_um, dtype=np.float64)
    edges = np.sqrt(lam[1:] * lam[:-1])
    edges = np.concatenate([[lam[0] ** 2 / edges[0]], edges, [lam[-1] ** 2 / edges[-1]]])
    shape = 1.0 / (lam ** 5 * np.expm1(14387.768775039337 / (lam * t_star)))
    spec = shape * np.diff(edges)
    return total * spec / spec.sum()


def panchromatic_disk(n_cells=64, n_lambda=24, n_pix=64, n_packets_total=2_400_000, face_on_tau_v=0.5,
                      emission_scale=1e11, channels=1) -> Problem:
    """The disk galaxy over a panchromatic wavelength grid (Sect. 2.1, 2.2):
    ``n_lambda`` wavelengths log-spaced from 0.1 to 1000 um, the stars a
    5800 K blackbody of unit total luminosity, synthetic optics without
    scattering far in the infrared (panchromatic_optics), three frames at 0,
    60 and 90 degrees and an SED instrument at 60 degrees.  ``emission_scale``
    (meta) is the dust emission's scale S for rt_dust_temperature: chosen so
    that the dust of this model settles at a few tens of kelvin."""
    base = disk_galaxy(n_cells=n_cells, n_lambda=3, n_pix=n_pix, face_on_tau_v=face_on_tau_v, channels=channels)
    wl = np.geomspace(0.1, 1000.0, n_lambda)
    kappa, albedo, g = panchromatic_optics(wl, face_on_tau_v / (2.0 * 0.2))
    src = replace(base.sources[0], lum=stellar_spectrum(wl))
    instr = base.instruments + [sed_instrument(60.0, channels=channels)]
    return replace(base, name=f"panchromatic_disk_{n_cells}", wavelengths=wl, kappa=kappa, albedo=albedo, g=g,
                   sources=[src], instruments=instr, run=Run(n_per_lambda=max(1, n_packets_total // n_lambda)),
                   meta={"emission_scale": float(emission_scale), "t_star": 5800.0})


def lognormal_cube(n_cells=64, sigma_ln=1.0, mean_axis_tau=2.0, smooth_cells=2.0, seed=4,
                   albedo=0.5, g=0.6, n_pix=128, n_packets=10_000_000, max_events=20) -> Problem:
    """Log-normal density on [-1, 1]^3: G = Gaussian-smoothed white noise,
    rho = exp(sigma_ln G / std(G)), scaled so that the mean full-axis column
    optical depth (kappa = 1) is ``mean_axis_tau``.  Central point source,
    face-on bilinear frame, termination after ``max_events`` events only."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n_cells,) * 3)
    G = gaussian_filter(noise, smooth_cells, mode="wrap")
    rho = np.exp(sigma_ln * G / G.std())
    dz = 2.0 / n_cells
    column = rho.sum(axis=0) * dz  # kappa = 1
    rho *= mean_axis_tau / column.mean()
    return Problem(
        name=f"lognormal_cube_{n_cells}",
        grid=cartesian_grid([-1.0, 1.0] * 3, rho.astype(np.float32)),
        wavelengths=_f64([0.55]), kappa=_f64([1.0]), albedo=_f64([albedo]), g=_f64([g]),
        sources=[Source("point", (0.0, 0.0, 0.0), _f64([1.0]))],
        instruments=[face_on(n_pix, 1.0, bilinear=True)],
        run=Run(n_per_lambda=n_packets, max_events=max_events, weight_cut=False),
        meta={"seed": seed},
    )


def batch_models(n_models=4096, seed=5, n_pix=64, packets=(1e4, 1e6), sides=(8, 48), axis_tau=(0.1, 20.0),
                 g=(0.0, 0.9), albedo=(0.3, 0.8)) -> list:
    """Many small one-wavelength models for a batched launch (the parameter
    searches of model fitting, Sect. 1).  Per model, drawn with
    ``default_rng(seed)``: cells per side uniform in ``sides`` (inclusive) on
    [-1, 1]^3; half the models (a random half) uniform, the others an
    exponential slab rho ~ exp(-|z| / (0.2 side)) with side = 2 the cube's
    side length, at cell centres; the optical depth along the full x axis
    through the centre (the central row of cells, kappa = 1) log-uniform in
    ``axis_tau``; g and the albedo uniform in their ranges; a central point
    source of unit luminosity; one ``n_pix``^2 face-on frame covering the
    cube; packets log-uniform in ``packets``."""
    rng = np.random.default_rng(seed)
    n_side = rng.integers(sides[0], sides[1] + 1, n_models)
    slab = rng.permutation(np.arange(n_models) < n_models // 2)
    taus = np.exp(rng.uniform(np.log(axis_tau[0]), np.log(axis_tau[1]), n_models))
    gs = rng.uniform(g[0], g[1], n_models)
    albs = rng.uniform(albedo[0], albedo[1], n_models)
    pk = np.rint(np.exp(rng.uniform(np.log(packets[0]), np.log(packets[1]), n_models))).astype(np.int64)
    bounds = [-1.0, 1.0] * 3
    out = []
    for m in range(n_models):
        side = int(n_side[m])
        if slab[m]:
            _, _, zs = cell_centres(bounds, (side, side, side))
            dens = np.broadcast_to(np.exp(-np.abs(zs) / (0.2 * 2.0))[:, None, None], (side, side, side))
        else:
            dens = np.ones((side, side, side))
        column = dens[side // 2, side // 2, :].sum() * (2.0 / side)
        dens = np.ascontiguousarray(dens * (taus[m] / column), dtype=np.float32)
        out.append(Problem(
            name=f"batch_model_{m}",
            grid=cartesian_grid(bounds, dens),
            wavelengths=_f64([0.55]), kappa=_f64([1.0]), albedo=_f64([albs[m]]), g=_f64([gs[m]]),
            sources=[Source("point", (0.0, 0.0, 0.0), _f64([1.0]))],
            instruments=[face_on(n_pix, 1.0)],
            run=Run(n_per_lambda=int(pk[m])),
            meta={"model": m, "slab": bool(slab[m]), "axis_tau": float(taus[m])},
        ))
    return out


def with_density(problem: Problem, density) -> Problem:
    """Copy of ``problem`` with a different density array (same grid shape)."""
    grid = replace(problem.grid, density=np.ascontiguousarray(density, dtype=np.float32))
    return replace(problem, grid=grid)


def with_packets(problem: Problem, n_per_lambda: int) -> Problem:
    return replace(problem, run=replace(problem.run, n_per_lambda=int(n_per_lambda)))


# ---------------------------------------------------------------- octrees
def build_octree(bounds, refine, leaf_value, max_level):
    """Octree by recursive 2x2x2 subdivision (Sect. 2.4), built level by level.

    ``refine(lo, hi, level) -> bool[N]`` decides which of N nodes (boxes
    lo[N, 3], hi[N, 3]) are split; nodes at ``max_level`` are never split.
    ``leaf_value(lo, hi) -> float[N]`` gives the density of leaves.  Returns a
    :class:`Grid` with ``child`` (int32 per node: first child index, children
    contiguous in octant order bit0 = x upper, bit1 = y upper, bit2 = z upper;
    or -(leaf + 1)) and per-leaf density, plus the leaf boxes."""
    b = np.asarray(bounds, dtype=np.float64)
    lo = b[[0, 2, 4]][None, :].copy()
    hi = b[[1, 3, 5]][None, :].copy()
    child_parts, leaf_lo, leaf_hi = [], [], []
    n_nodes_before = 0
    n_leaves = 0
    level = 0
    octs = np.array([[(o >> a) & 1 for a in range(3)] for o in range(8)], dtype=np.float64)
    while lo.shape[0]:
        n = lo.shape[0]
        split = np.zeros(n, dtype=bool) if level >= max_level else np.asarray(refine(lo, hi, level), dtype=bool)
        child = np.empty(n, dtype=np.int64)
        n_split = int(split.sum())
        first_next = n_nodes_before + n
        child[split] = first_next + 8 * np.arange(n_split)
        leaf_ids = n_leaves + np.arange(n - n_split)
        child[~split] = -(leaf_ids + 1)
        n_leaves += n - n_split
        child_parts.append(child)
        leaf_lo.append(lo[~split])
        leaf_hi.append(hi[~split])
        plo, phi = lo[split], hi[split]
        mid = 0.5 * (plo + phi)
        upper = np.tile(octs, (n_split, 1)) > 0
        clo = np.where(upper, np.repeat(mid, 8, axis=0), np.repeat(plo, 8, axis=0))
        chi = np.where(upper, np.repeat(phi, 8, axis=0), np.repeat(mid, 8, axis=0))
        n_nodes_before += n
        lo, hi = clo, chi
        level += 1
    child = np.concatenate(child_parts)
    if child.max(initial=0) > np.iinfo(np.int32).max or n_leaves > np.iinfo(np.int32).max:
        raise ValueError("octree too large for int32 node indices")
    llo = np.concatenate(leaf_lo)
    lhi = np.concatenate(leaf_hi)
    dens = np.asarray(leaf_value(llo, lhi), dtype=np.float32)
    g = Grid("octree", _f64(bounds), np.ascontiguousarray(dens), child.astype(np.int32))
    return g, llo, lhi


def build_bintree(bounds, refine, leaf_value, max_depth, axis_of=None):
    """k-d tree by recursive halving of boxes (Table 1(d): BinTree), built
    level by level.  ``axis_of(lo, hi, depth) -> int[N]`` gives the split
    axis of each node (default: the axes in turn, z, y, x, z, ..., i.e. the
    order of the bits of a Morton key from the top); ``refine`` and
    ``leaf_value`` as for :func:`build_octree`.  Returns (Grid, leaf lo,
    leaf hi)."""
    b = np.asarray(bounds, dtype=np.float64)
    lo = b[[0, 2, 4]][None, :].copy()
    hi = b[[1, 3, 5]][None, :].copy()
    child_parts, axis_parts, leaf_lo, leaf_hi = [], [], [], []
    n_before = 0
    n_leaves = 0
    depth = 0
    while lo.shape[0]:
        n = lo.shape[0]
        split = np.zeros(n, dtype=bool) if depth >= max_depth else np.asarray(refine(lo, hi, depth), dtype=bool)
        axis = (np.full(n, 2 - depth % 3) if axis_of is None else np.asarray(axis_of(lo, hi, depth))).astype(np.int8)
        child = np.empty(n, dtype=np.int64)
        n_split = int(split.sum())
        child[split] = n_before + n + 2 * np.arange(n_split)
        child[~split] = -(n_leaves + np.arange(n - n_split) + 1)
        n_leaves += n - n_split
        child_parts.append(child)
        axis_parts.append(np.where(split, axis, 0).astype(np.int8))
        leaf_lo.append(lo[~split])
        leaf_hi.append(hi[~split])
        plo, phi, pax = lo[split], hi[split], axis[split].astype(np.int64)
        mid = 0.5 * (plo[np.arange(n_split), pax] + phi[np.arange(n_split), pax])
        clo = np.repeat(plo, 2, axis=0)
        chi = np.repeat(phi, 2, axis=0)
        rows = np.arange(n_split)
        chi[2 * rows, pax] = mid       # lower child
        clo[2 * rows + 1, pax] = mid   # upper child
        n_before += n
        lo, hi = clo, chi
        depth += 1
    child = np.concatenate(child_parts)
    if child.max(initial=0) > np.iinfo(np.int32).max or n_leaves > np.iinfo(np.int32).max:
        raise ValueError("k-d tree too large for int32 node indices")
    llo, lhi = np.concatenate(leaf_lo), np.concatenate(leaf_hi)
    dens = np.asarray(leaf_value(llo, lhi), dtype=np.float32)
    g = Grid("bintree", _f64(bounds), np.ascontiguousarray(dens), child.astype(np.int32),
             split_axis=np.concatenate(axis_parts))
    return g, llo, lhi


def voronoi_grid(bounds, sites, density, mirror_depth=3.0) -> Grid:
    """Voronoi grid (Table 1(d): VoronoiDustGrid; Sect. 2.4): cell c is the
    part of the domain nearer to ``sites[c]`` than to any other site.  The
    neighbour lists come from a Delaunay triangulation (scipy) of the sites
    and of their mirror images across each domain face for the sites within
    ``mirror_depth`` mean spacings of it.  A mirror image is never nearer
    than its site to a point inside the domain, so every pair of cells that
    share a face inside the domain stays a Delaunay pair and is listed; the
    images only remove pairs whose common face lies outside.  A listed pair
    without a face inside the domain costs a walk one plane test and
    changes nothing.  Sites must lie strictly inside the domain."""
    from scipy.spatial import Delaunay
    b = np.asarray(bounds, dtype=np.float64).reshape(3, 2)
    sites = np.ascontiguousarray(sites, dtype=np.float64)
    n = len(sites)
    if not np.all((sites > b[:, 0]) & (sites < b[:, 1])):
        raise ValueError("Voronoi sites must lie strictly inside the domain")
    h = mirror_depth * (np.prod(b[:, 1] - b[:, 0]) / n) ** (1.0 / 3.0)
    pts = [sites]
    for a in range(3):
        for wall in b[a]:
            near = np.abs(sites[:, a] - wall) < h
            m = sites[near].copy()
            m[:, a] = 2.0 * wall - m[:, a]
            pts.append(m)
    indptr, indices = Delaunay(np.concatenate(pts)).vertex_neighbor_vertices
    row = np.repeat(np.arange(n), np.diff(indptr[:n + 1]))
    col = indices[:indptr[n]]
    keep = col < n
    row, col = row[keep], col[keep]
    order = np.lexsort((col, row))
    counts = np.bincount(row, minlength=n)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return Grid("voronoi", _f64(bounds), np.ascontiguousarray(density, dtype=np.float32).ravel(),
                child=col[order].astype(np.int32), sites=sites, offsets=offsets)


def voronoi_lattice(grid: Grid) -> Grid:
    """The Voronoi grid whose sites are the cell centres of a cartesian grid
    (row-major order), with the six face neighbours of every cell as its
    neighbour lists: its cells are the cartesian cells, so transport on it
    must equal transport on the cartesian grid."""
    nx, ny, nz = grid.shape
    xs, ys, zs = cell_centres(grid.bounds, (nx, ny, nz))
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    sites = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    iz, iy, ix = (a.ravel() for a in np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij"))
    cols = []
    for (dx, dy, dz) in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
        jx, jy, jz = ix + dx, iy + dy, iz + dz
        ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
        cols.append(np.where(ok, jx + nx * (jy + ny * jz), -1))
    cols = np.stack(cols, axis=1)
    counts = (cols >= 0).sum(axis=1)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return Grid("voronoi", _f64(grid.bounds), np.ascontiguousarray(grid.density, dtype=np.float32).ravel(),
                child=cols[cols >= 0].astype(np.int32), sites=sites, offsets=offsets)


def voronoi_disk(n_sites=20_000, n_lambda=3, n_pix=64, n_packets_total=60_000, face_on_tau_v=0.5, seed=7,
                 uniform_fraction=0.1, channels=1) -> Problem:
    """The disk galaxy (:func:`disk_galaxy`: domain, stars, optics, frames at
    0, 60 and 90 degrees) on a Voronoi grid whose sites are drawn from its
    dust density, as in the Voronoi grid of the paper's grid figure (Sect.
    2.4): radius R from the exponential disk's surface density (R e^{-R/6}),
    |z| exponential with scale 0.2 kpc, a uniform share ``uniform_fraction``
    over the whole domain; each cell takes the density at its site."""
    bounds = [-25.0, 25.0, -25.0, 25.0, -3.0, 3.0]
    rng = np.random.default_rng(seed)
    n_uniform = int(round(uniform_fraction * n_sites))
    parts, have = [], 0
    while have < n_sites - n_uniform:
        m = 2 * (n_sites - n_uniform - have) + 16
        R = rng.gamma(2.0, 6.0, m)
        phi = rng.uniform(0.0, 2.0 * math.pi, m)
        z = rng.laplace(0.0, 0.2, m)
        p = np.stack([R * np.cos(phi), R * np.sin(phi), z], axis=1)
        p = p[(np.abs(p[:, 0]) < 25.0) & (np.abs(p[:, 1]) < 25.0) & (np.abs(p[:, 2]) < 3.0)]
        parts.append(p[:n_sites - n_uniform - have])
        have += len(parts[-1])
    lo, hi = np.array([-25.0, -25.0, -3.0]), np.array([25.0, 25.0, 3.0])
    parts.append(lo + rng.uniform(0.0, 1.0, (n_uniform, 3)) * (hi - lo))
    sites = np.concatenate(parts)
    R = np.hypot(sites[:, 0], sites[:, 1])
    dens = np.exp(-R / 6.0 - np.abs(sites[:, 2]) / 0.2)
    wl = np.geomspace(0.15, 2.2, n_lambda)
    kappa, albedo, g = synthetic_optics(wl, face_on_tau_v / (2.0 * 0.2))
    instr = [Instrument(math.radians(inc), -math.pi / 2, 0.0, n_pix, n_pix, 25.0, 25.0, channels=channels)
             for inc in (0.0, 60.0, 90.0)]
    grid = voronoi_grid(bounds, sites, dens)
    return Problem(
        name=f"voronoi_disk_{n_sites}",
        grid=grid, wavelengths=wl, kappa=kappa, albedo=albedo, g=g,
        sources=[Source("expdisk", (0.0, 0.0, 0.0), np.ones(n_lambda), scale_r=4.0, scale_z=0.35)],
        instruments=instr,
        run=Run(n_per_lambda=max(1, int(n_packets_total) // n_lambda)),
        meta={"sites": n_sites, "neighbours_per_cell": float(grid.child.size) / n_sites, "seed": seed},
    )


def octree_problem_like(problem: Problem, grid: Grid) -> Problem:
    return replace(problem, grid=grid)


def _spread3(v):
    """Interleave the low 10 bits of v with two zero bits each (Morton order)."""
    v = v.astype(np.uint64) & np.uint64(0x3FF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x30000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x300F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x9249249)
    return v


def _clumpy_samples(n_particles, n_samples, max_level, seed, half, chunk):
    """Gaussian dust clumps and the Morton keys (max_level bits per axis) of
    n_samples points drawn from their mass, sorted; the clumps' centres from
    a double-exponential dust disk (h_R = 6, h_z = 0.2 kpc), widths
    log-uniform in 20-200 pc, masses log-normal (sigma_ln = 1.5), total 1.
    Returns (keys, kept): samples outside the box are dropped."""
    rng = np.random.default_rng(seed)
    R = rng.gamma(2.0, 6.0, n_particles)
    ph = rng.uniform(0.0, 2 * math.pi, n_particles)
    cx, cy = R * np.cos(ph), R * np.sin(ph)
    cz = rng.laplace(0.0, 0.2, n_particles)
    sig = np.exp(rng.uniform(math.log(0.02), math.log(0.2), n_particles))
    mass = rng.lognormal(0.0, 1.5, n_particles)
    mass /= mass.sum()
    cum = np.cumsum(mass)
    n_side = 1 << max_level
    keys = []
    kept = 0
    for start in range(0, n_samples, chunk):
        m = min(chunk, n_samples - start)
        idx = np.minimum(np.searchsorted(cum, rng.uniform(0.0, cum[-1], m)), n_particles - 1)
        s = sig[idx]
        px = cx[idx] + s * rng.standard_normal(m)
        py = cy[idx] + s * rng.standard_normal(m)
        pz = cz[idx] + s * rng.standard_normal(m)
        inside = (np.abs(px) < half) & (np.abs(py) < half) & (np.abs(pz) < half)
        ix = ((px[inside] + half) * (n_side / (2 * half))).astype(np.int64).clip(0, n_side - 1)
        iy = ((py[inside] + half) * (n_side / (2 * half))).astype(np.int64).clip(0, n_side - 1)
        iz = ((pz[inside] + half) * (n_side / (2 * half))).astype(np.int64).clip(0, n_side - 1)
        keys.append((_spread3(ix) | (_spread3(iy) << np.uint64(1)) | (_spread3(iz) << np.uint64(2))).astype(np.uint32))
        kept += int(inside.sum())
    return np.sort(np.concatenate(keys)), kept


def _prefix_counts(keys, n_bits, depths):
    """Sample counts per key prefix: for each depth d the distinct values of
    keys >> (n_bits - d) and their counts (runs of the sorted keys)."""
    out_k, out_c = [], []
    for d in depths:
        k = keys >> np.uint32(n_bits - d)
        starts = np.flatnonzero(np.concatenate(([True], k[1:] != k[:-1])))
        out_k.append(k[starts])
        out_c.append(np.diff(np.append(starts, len(k))))
    return out_k, out_c


def clumpy_bintree(n_particles=20_000, n_samples=400_000, target_leaves=20_000, max_level=7, seed=3, n_lambda=4,
                   n_pix=64, n_packets_total=80_000, half=20.0, chunk=10_000_000, channels=1):
    """The clumpy medium of :func:`clumpy_octree` on a k-d tree (Table 1(d):
    BinTree): nodes halved along z, y, x in turn (the bits of a Morton key
    from the top), refined while their sampled mass exceeds delta M_tot, up
    to 3 max_level splits; delta chosen by bisection for about
    ``target_leaves`` leaves."""
    keys, kept = _clumpy_samples(n_particles, n_samples, max_level, seed, half, chunk)
    n_bits = 3 * max_level
    weight = 1.0 / n_samples
    lk, lc = _prefix_counts(keys, n_bits, range(n_bits + 1))

    def n_leaves(thr):
        return 1 + sum(int((lc[d] > thr).sum()) for d in range(n_bits))
    lo_t, hi_t = 0.0, float(lc[0].max())
    for _ in range(60):
        mid = 0.5 * (lo_t + hi_t)
        if n_leaves(mid) > target_leaves:
            lo_t = mid
        else:
            hi_t = mid
    thr = hi_t
    n_side = 1 << max_level

    def count_of(lo, depth):
        cell = np.rint((lo + half) / (2 * half) * n_side).astype(np.int64)
        full = _spread3(cell[:, 0]) | (_spread3(cell[:, 1]) << np.uint64(1)) | (_spread3(cell[:, 2]) << np.uint64(2))
        k = (full >> np.uint64(n_bits - depth)).astype(np.uint32)
        u, c = lk[depth], lc[depth]
        pos = np.searchsorted(u, k)
        pos_c = np.minimum(pos, len(u) - 1)
        return np.where((pos < len(u)) & (u[pos_c] == k), c[pos_c], 0)

    def leaf_value(lo, hi):
        vol = np.prod(hi - lo, axis=1)
        depth = np.rint(np.log2((2 * half) ** 3 / vol)).astype(np.int64)
        out = np.zeros(len(lo))
        for d in np.unique(depth):
            sel = depth == d
            out[sel] = count_of(lo[sel], int(d)) * weight / vol[sel]
        return out

    grid, _, _ = build_bintree([-half, half] * 3, lambda lo, hi, d: count_of(lo, d) > thr, leaf_value, n_bits)
    wl = np.geomspace(0.15, 2.2, n_lambda)
    kappa, albedo, g = synthetic_optics(wl, 0.5 * 2 * math.pi * 6.0 ** 2)
    instr = [Instrument(math.radians(inc), -math.pi / 2, 0.0, n_pix, n_pix, half, half, channels=channels)
             for inc in (0.0, 90.0)]
    return Problem(
        name=f"clumpy_bintree_{grid.n_cells}",
        grid=grid, wavelengths=wl, kappa=kappa, albedo=albedo, g=g,
        sources=[Source("plummer", (0.0, 0.0, 0.0), np.full(n_lambda, 0.3), scale_r=1.0),
                 Source("expdisk", (0.0, 0.0, 0.0), np.full(n_lambda, 0.7), scale_r=4.0, scale_z=0.35)],
        instruments=instr,
        run=Run(n_per_lambda=max(1, int(n_packets_total) // n_lambda)),
        meta={"delta": thr * weight, "leaves": grid.n_cells, "nodes": int(grid.child.size),
              "samples_inside": kept, "seed": seed},
    )


def clumpy_octree(n_particles=1_000_000, n_samples=100_000_000, target_leaves=5_000_000, max_level=10, seed=3,
                  n_lambda=20, n_pix=1024, n_packets_total=200_000_000, half=20.0, chunk=10_000_000, channels=1):
    """Clumpy dust on an adaptive octree (Sect. 2.4).

    ``n_particles`` Gaussian clumps: centres drawn from a double-exponential
    dust disk (h_R = 6 kpc, h_z = 0.2 kpc), widths log-uniform in 20-200 pc,
    masses log-normal (sigma_ln = 1.5), total mass 1.  The mixture is binned
    by drawing ``n_samples`` points from it (Morton keys at ``max_level``); a
    node is refined while its mass exceeds delta * M_tot, with delta chosen by
    bisection so that the tree has about ``target_leaves`` leaves.  Leaf
    density = binned mass / leaf volume.  kappa_V makes the equivalent smooth
    disk's face-on central optical depth 0.5.  Sources: Plummer bulge
    (a = 1 kpc, 30 %) and exponential disk (h_R = 4, h_z = 0.35 kpc, 70 %).
    Two ``n_pix``^2 frames at inclinations 0 and 90 degrees."""
    if max_level > 10:
        raise ValueError("max_level <= 10 (30-bit Morton keys)")
    keys, kept = _clumpy_samples(n_particles, n_samples, max_level, seed, half, chunk)
    weight = 1.0 / n_samples  # mass per sample (M_tot = 1, outside samples dropped)
    # sample counts per node at every level
    level_keys, level_counts = _prefix_counts(keys, 3 * max_level, [3 * L for L in range(max_level + 1)])
    # threshold in samples: leaves = 1 + 7 * (#nodes above threshold at levels < max_level)
    def n_leaves(thr):
        return 1 + 7 * sum(int((level_counts[L] > thr).sum()) for L in range(max_level))
    lo_t, hi_t = 0.0, float(level_counts[0].max())
    for _ in range(60):
        mid = 0.5 * (lo_t + hi_t)
        if n_leaves(mid) > target_leaves:
            lo_t = mid
        else:
            hi_t = mid
    thr = hi_t

    def key_of(lo, level):
        cell = np.rint((lo + half) / (2 * half) * (1 << level)).astype(np.int64)
        return (_spread3(cell[:, 0]) | (_spread3(cell[:, 1]) << np.uint64(1)) | (_spread3(cell[:, 2]) << np.uint64(2)))

    def count_of(lo, level):
        k = key_of(lo, level)
        u, c = level_keys[level], level_counts[level]
        pos = np.searchsorted(u, k)
        pos_c = np.minimum(pos, len(u) - 1)
        return np.where((pos < len(u)) & (u[pos_c] == k), c[pos_c], 0)

    level_of = {}

    def refine(lo, hi, level):
        return count_of(lo, level) > thr

    def leaf_value(lo, hi):
        size = hi[:, 0] - lo[:, 0]
        level = np.rint(np.log2(2 * half / size)).astype(np.int64)
        out = np.zeros(len(lo))
        for L in np.unique(level):
            sel = level == L
            out[sel] = count_of(lo[sel], int(L)) * weight / (size[sel] ** 3)
        return out

    grid, llo, lhi = build_octree([-half, half] * 3, refine, leaf_value, max_level)
    wl = np.geomspace(0.15, 2.2, n_lambda)
    kappa, albedo, g = synthetic_optics(wl, 0.5 * 2 * math.pi * 6.0 ** 2)
    instr = [Instrument(math.radians(inc), -math.pi / 2, 0.0, n_pix, n_pix, half, half, channels=channels)
             for inc in (0.0, 90.0)]
    return Problem(
        name=f"clumpy_octree_{grid.n_cells}",
        grid=grid, wavelengths=wl, kappa=kappa, albedo=albedo, g=g,
        sources=[Source("plummer", (0.0, 0.0, 0.0), np.full(n_lambda, 0.3), scale_r=1.0),
                 Source("expdisk", (0.0, 0.0, 0.0), np.full(n_lambda, 0.7), scale_r=4.0, scale_z=0.35)],
        instruments=instr,
        run=Run(n_per_lambda=max(1, int(n_packets_total) // n_lambda)),
        meta={"delta": thr * weight, "leaves": grid.n_cells, "nodes": int(grid.child.size),
              "samples_inside": kept, "seed": seed},
    )
