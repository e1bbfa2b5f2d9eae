"""Seeded synthetic instruments shaped like the paper's three test problems.

This module only *describes* instruments as plain data (component lists, the
mu(E) material tables and the voxel phantom bytes).  It holds none of the
tracing arithmetic: both the CUDA path and the CPU oracle consume these
descriptions through their own, independent marshalling code.

Units: positions and lengths in metres, energies in keV, attenuation
coefficients in 1/m.  Every component dict has

    type         one of COMPONENT_TYPES
    pos          (x, y, z) of the component origin in the frame of `relative_to`
    rot          row-major 3x3 rotation (local -> parent), or None for identity
    relative_to  index of an earlier component, or -1 for the lab frame

plus the type-specific keys documented in COMPONENT_TYPES.  Component 0 is
always the source.

Workload shapes follow the paper's instruments: a flat-spectrum source with a
slit and position/energy monitors (Sec. 3.1, Sec. 3.2), a bremsstrahlung
(Kramers-law) tube spectrum through an absorbing sample into an
energy-resolved detector, and a voxelised multi-material phantom in the
energy-dispersive CT geometry of Sec. 3.3.  The paper's tungsten, water and
beryllium tables are not available; synthetic mu(E) = a E^-3 (x jump above a
K-edge) + b materials stand in for them.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MM = 1e-3

# type name -> required parameter keys (besides type/pos/rot/relative_to)
COMPONENT_TYPES = {
    # shape: "disk" (radius) | "point" | "rect" (spot_w, spot_h) | "gauss"
    # (sigma_x, sigma_y; optional divergence sigmas div_x, div_y weight the
    # ray); spectrum: "flat" (uniform in [e_min, e_max)) | "kramers"
    # ((e0 - E)/E, e0 = tube kVp) | "gauss" (e0, sigma_e); directions aim at
    # a uniform point of a target_w x target_h rectangle centred on the local
    # z axis at distance target_dist.
    "source": ("shape", "spectrum", "e_min", "e_max", "target_dist",
               "target_w", "target_h"),
    "slit_rect": ("xmin", "xmax", "ymin", "ymax"),
    "slit_circ": ("radius",),
    # absorbers attenuate the weight by exp(-mu(E) L) over the chord L;
    # the ray keeps its line.  Box: full widths; cylinder axis = local y.
    "abs_box": ("wx", "wy", "wz", "material"),
    "abs_cyl": ("radius", "height", "material"),
    "abs_sphere": ("radius", "material"),
    # voxel phantom centred on the origin; bytes are material indices;
    # optional march = steps per voxel (the paper's fixed-step traversal) and,
    # with it, scatter=True (the instrument's mu_scatter per material)
    "phantom": ("nx", "ny", "nz", "voxel"),
    # monitors are non-absorbing detectors in the local z = 0 plane; with the
    # optional restore=True the ray leaves a monitor as it entered it
    "mon_psd": ("nx", "ny", "xmin", "xmax", "ymin", "ymax"),
    "mon_e": ("ne", "e_min", "e_max", "xmin", "xmax", "ymin", "ymax"),
    "mon_l": ("nl", "l_min", "l_max", "xmin", "xmax", "ymin", "ymax"),
    "mon_epsd": ("nx", "ny", "ne", "xmin", "xmax", "ymin", "ymax",
                 "e_min", "e_max"),
    # compound refractive lens: n_lenses double-sided parabolic lenses of
    # apex radius `radius`, apex thickness `thickness` and aperture radius
    # `aperture`, centred `pitch` apart along local z; refractive index
    # 1 - delta0 (e_ref / E)^2; the lens material attenuates
    "lens_parab": ("radius", "thickness", "aperture", "n_lenses", "delta0", "e_ref", "pitch",
                   "material"),
}

MONITOR_TYPES = ("mon_psd", "mon_e", "mon_l", "mon_epsd")


def monitor_bins(comp: dict) -> int:
    """Number of bins of a monitor component (0 for other types)."""
    t = comp["type"]
    if t == "mon_psd":
        return comp["nx"] * comp["ny"]
    if t == "mon_e":
        return comp["ne"]
    if t == "mon_l":
        return comp["nl"]
    if t == "mon_epsd":
        return comp["nx"] * comp["ny"] * comp["ne"]
    return 0


def rot_y(theta: float) -> tuple:
    """Row-major rotation by `theta` radians about the y axis."""
    c, s = math.cos(theta), math.sin(theta)
    return (c, 0.0, s, 0.0, 1.0, 0.0, -s, 0.0, c)


@dataclass
class Materials:
    """Per-cell linear attenuation tables: on cell j of [e_min, e_max),
    mu_m(E) = coef[m, j, 0] + coef[m, j, 1] * E  (1/m, E in keV)."""
    e_min: float
    e_max: float
    coef: np.ndarray  # float64 [n_mat, n_cell, 2]

    @property
    def n_mat(self) -> int:
        return int(self.coef.shape[0])

    @property
    def n_cell(self) -> int:
        return int(self.coef.shape[1])


@dataclass
class Instrument:
    components: list
    materials: Materials | None = None
    phantom: np.ndarray | None = None  # uint8 [nz, ny, nx], x fastest
    # Rayleigh (elastic) and Compton scattering coefficients (1/m) of a
    # scattering phantom: one value per material, or per-cell linear tables
    # shaped like materials.coef (tabulate_curves)
    mu_scatter: np.ndarray | None = None
    mu_compton: np.ndarray | None = None
    instr_id: int = 0
    name: str = ""
    meta: dict = field(default_factory=dict)


def component(type_: str, pos=(0.0, 0.0, 0.0), rot=None, relative_to=-1, **params) -> dict:
    if type_ not in COMPONENT_TYPES:
        raise ValueError(f"unknown component type {type_!r}")
    missing = [k for k in COMPONENT_TYPES[type_] if k not in params]
    if missing:
        raise ValueError(f"{type_}: missing parameters {missing}")
    d = {"type": type_, "pos": tuple(float(v) for v in pos),
         "rot": None if rot is None else tuple(float(v) for v in rot),
         "relative_to": int(relative_to)}
    d.update(params)
    return d


# ---------------------------------------------------------------- materials
def tabulate_materials(params, e_min: float, e_max: float, n_cell: int) -> Materials:
    """Tabulate mu(E) = a E^-3 * (jump if E >= edge) + b for each material.

    `params` is a list of (a [keV^3/m], b [1/m], edge [keV] or None, jump).
    Each cell's line passes through the one-sided limits of mu at its two
    ends, so an edge that falls on a cell boundary is represented exactly.
    """
    de = (e_max - e_min) / n_cell
    coef = np.zeros((len(params), n_cell, 2), dtype=np.float64)
    j = np.arange(n_cell, dtype=np.float64)
    e_lo = e_min + j * de
    e_hi = e_min + (j + 1) * de
    for m, (a, b, edge, jump) in enumerate(params):
        def mu(e, right_side):
            f = np.ones_like(e)
            if edge is not None:
                f = np.where((e > edge) | ((e == edge) & right_side), jump, 1.0)
            return a * f / e**3 + b
        mu_lo = mu(e_lo, True)    # right-hand limit at the cell's lower end
        mu_hi = mu(e_hi, False)   # left-hand limit at the cell's upper end
        slope = (mu_hi - mu_lo) / de
        coef[m, :, 0] = mu_lo - slope * e_lo
        coef[m, :, 1] = slope
    return Materials(e_min=e_min, e_max=e_max, coef=coef)


def tabulate_curves(curves, e_min: float, e_max: float, n_cell: int) -> np.ndarray:
    """Per-cell linear tables [n_mat, n_cell, 2] (the layout of
    Materials.coef) of smooth curves: each cell's line passes through the
    material's curve f(E) (1/m, a callable of E in keV) at the cell's two
    ends."""
    de = (e_max - e_min) / n_cell
    j = np.arange(n_cell, dtype=np.float64)
    e_lo, e_hi = e_min + j * de, e_min + (j + 1) * de
    out = np.zeros((len(curves), n_cell, 2))
    for m, f in enumerate(curves):
        lo, hi = f(e_lo), f(e_hi)
        slope = (hi - lo) / de
        out[m, :, 0] = lo - slope * e_lo
        out[m, :, 1] = slope
    return out


ME_C2 = 510.99895              # electron rest energy, keV
R_E = 2.8179403262e-15         # classical electron radius, m
WATER_NE = 3.3429e29           # electrons per m^3 of water (1 g/cm^3, 10 per 18.015 g/mol)


def klein_nishina_sigma(E):
    """Total Klein-Nishina cross-section of a free electron (m^2) at photon
    energy E (keV), the textbook closed form with k = E / m_e c^2:
    2 pi r_e^2 [ (1+k)/k^2 (2(1+k)/(1+2k) - ln(1+2k)/k) + ln(1+2k)/(2k)
    - (1+3k)/(1+2k)^2 ]."""
    k = np.asarray(E, dtype=np.float64) / ME_C2
    lg = np.log1p(2.0 * k)
    return 2.0 * math.pi * R_E ** 2 * ((1.0 + k) / k ** 2 * (2.0 * (1.0 + k) / (1.0 + 2.0 * k) - lg / k)
                                       + lg / (2.0 * k) - (1.0 + 3.0 * k) / (1.0 + 2.0 * k) ** 2)


def water_scattering(scale=(0.0, 1.0, 2.0), e_min: float = 20.0, e_max: float = 120.0,
                     n_cell: int = 500, rayleigh_40: float = 1.2):
    """Synthetic energy-dependent scattering tables of water-like materials
    (material m is `scale[m]` x water): Compton = the free-electron
    Klein-Nishina coefficient WATER_NE sigma_KN(E) (22.2 /m in the Thomson
    limit, 19.3 /m at 40 keV, 16.5 /m at 100 keV); Rayleigh falling as
    E^-2 from `rayleigh_40` /m at 40 keV.  Returns (mu_scatter, mu_compton),
    each [n_mat, n_cell, 2] on the cells of the attenuation tables."""
    ray = [lambda e, s=s: s * rayleigh_40 * (40.0 / e) ** 2 for s in scale]
    com = [lambda e, s=s: s * WATER_NE * klein_nishina_sigma(e) for s in scale]
    return tabulate_curves(ray, e_min, e_max, n_cell), tabulate_curves(com, e_min, e_max, n_cell)


WATER_A = 5.12e5   # keV^3/m
WATER_B = 17.0     # 1/m

# the single material of the absorption instrument: a E^-3 + b with a x5
# K-edge jump at 60 keV (a = 1.6e4 keV^3/cm, b = 0.02 /cm)
ABS_MATERIAL = [(1.6e6, 2.0, 60.0, 5.0)]

# eight phantom materials: vacuum, a water-like background and six inclusions
# spread over 0.3x-30x water with K-edges at 33, 50, 69 and 88 keV
PHANTOM_MATERIALS = [
    (0.0, 0.0, None, 1.0),
    (WATER_A, WATER_B, None, 1.0),
    (0.3 * WATER_A, 0.6 * WATER_B, None, 1.0),
    (2.0 * WATER_A, 1.2 * WATER_B, None, 1.0),
    (6.0 * WATER_A, 2.0 * WATER_B, 33.0, 5.0),
    (10.0 * WATER_A, 3.0 * WATER_B, 50.0, 5.0),
    (20.0 * WATER_A, 5.0 * WATER_B, 69.0, 5.0),
    (30.0 * WATER_A, 8.0 * WATER_B, 88.0, 5.0),
]


# ---------------------------------------------------------------- phantom
def make_phantom(n: int = 256, seed: int = 3, n_spheres: int = 48, n_boxes: int = 16,
                 n_mat: int = 8) -> np.ndarray:
    """Seeded n^3 uint8 phantom: vacuum, a water-like box over the central 80 %
    of the cube, then random spheres and boxes of materials 2..n_mat-1
    painted in order.  Returned as [nz, ny, nx] (x fastest)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    vox = np.zeros((n, n, n), dtype=np.uint8)
    lo, hi = int(round(0.1 * n)), int(round(0.9 * n))
    vox[lo:hi, lo:hi, lo:hi] = 1
    rmin, rmax = max(1, n // 64), max(2, (n * 5) // 32)
    for _ in range(n_spheres):
        c = rng.uniform(lo, hi, size=3)
        r = rng.uniform(rmin, rmax)
        m = int(rng.integers(2, n_mat))
        a = np.maximum(np.floor(c - r).astype(int), 0)
        b = np.minimum(np.ceil(c + r).astype(int) + 1, n)
        zz, yy, xx = np.meshgrid(np.arange(a[2], b[2]), np.arange(a[1], b[1]),
                                 np.arange(a[0], b[0]), indexing="ij")
        inside = ((xx + 0.5 - c[0])**2 + (yy + 0.5 - c[1])**2
                  + (zz + 0.5 - c[2])**2) <= r * r
        sub = vox[a[2]:b[2], a[1]:b[1], a[0]:b[0]]
        sub[inside] = m
    for _ in range(n_boxes):
        size = rng.integers(max(1, n // 32), max(2, n // 4) + 1, size=3)
        corner = rng.integers(lo, max(lo + 1, hi - size.min()), size=3)
        m = int(rng.integers(2, n_mat))
        e = np.minimum(corner + size, n)
        vox[corner[2]:e[2], corner[1]:e[1], corner[0]:e[0]] = m
    return vox


# ---------------------------------------------------------------- configs
def flat_slit_instrument(slit_w: float = 0.5 * MM, instr_id: int = 0) -> Instrument:
    """Plain flat-spectrum instrument: disk source (radius 0.5 mm), energy
    uniform 10-30 keV, directions uniform onto a 1x1 mm target at 1 m; a
    square slit of side `slit_w` at 0.5 m; a 100x100-pixel PSD (2x2 mm) and a
    200-bin energy monitor (same aperture) at 1 m."""
    h = 0.5 * slit_w
    comps = [
        component("source", shape="disk", radius=0.5 * MM, spectrum="flat",
                  e_min=10.0, e_max=30.0, target_dist=1.0,
                  target_w=1.0 * MM, target_h=1.0 * MM),
        component("slit_rect", pos=(0, 0, 0.5), xmin=-h, xmax=h, ymin=-h, ymax=h),
        component("mon_psd", pos=(0, 0, 1.0), nx=100, ny=100,
                  xmin=-1 * MM, xmax=1 * MM, ymin=-1 * MM, ymax=1 * MM),
        component("mon_e", pos=(0, 0, 1.0), ne=200, e_min=10.0, e_max=30.0,
                  xmin=-1 * MM, xmax=1 * MM, ymin=-1 * MM, ymax=1 * MM),
    ]
    return Instrument(components=comps, instr_id=instr_id, name="flat_slit_1e6",
                      meta={"slit_w": slit_w})


def absorption_instrument(angle: float = 0.0, instr_id: int = 0, n_cell: int = 1000,
                          nx: int = 128, ne: int = 256, side: float = 25.6 * MM) -> Instrument:
    """Absorption instrument: point source, Kramers spectrum 20-120 keV, cone
    onto the 10x10 mm silhouette of a cylinder (radius 5 mm, height 10 mm,
    axis y, centred at 0.5 m, rotated by `angle` about its own axis) of the
    synthetic K-edge material; a 128x128-pixel (0.2 mm) x 256-energy-bin
    detector at 1 m (`side` wide, whatever the pixel count)."""
    half = 0.5 * side
    comps = [
        component("source", shape="point", spectrum="kramers", e_min=20.0,
                  e_max=120.0, e0=120.0, target_dist=0.5,
                  target_w=10 * MM, target_h=10 * MM),
        component("abs_cyl", pos=(0, 0, 0.5), rot=rot_y(angle) if angle else None,
                  radius=5 * MM, height=10 * MM, material=0),
        component("mon_epsd", pos=(0, 0, 1.0), nx=nx, ny=nx, ne=ne,
                  xmin=-half, xmax=half, ymin=-half, ymax=half,
                  e_min=20.0, e_max=120.0),
    ]
    mats = tabulate_materials(ABS_MATERIAL, 20.0, 120.0, n_cell)
    return Instrument(components=comps, materials=mats, instr_id=instr_id,
                      name="absorption_cyl_128x128x256", meta={"angle": angle})


def ct_instrument(angle: float = 0.0, n: int = 256, voxel: float = 0.5 * MM,
                  n_pix: int = 256, pix: float = 1.0 * MM, ne: int = 128,
                  window: float = 1.0, phantom_seed: int = 3, spot: float = 0.0,
                  instr_id: int = 0, phantom: np.ndarray | None = None) -> Instrument:
    """Energy-dispersive CT projection: point source (or a square focal spot of
    side `spot`), Kramers spectrum 20-160 keV, cone uniform onto a window of
    `window` x the detector side at 1 m; an n^3 voxel phantom (`voxel` m)
    centred at 0.5 m and rotated by `angle` about y; an n_pix^2 x ne
    energy-resolved detector at 1 m."""
    side = n_pix * pix
    half = 0.5 * side
    src = dict(spectrum="kramers", e_min=20.0, e_max=160.0, e0=160.0,
               target_dist=1.0, target_w=window * side, target_h=window * side)
    if spot > 0:
        src.update(shape="rect", spot_w=spot, spot_h=spot)
    else:
        src.update(shape="point")
    comps = [
        component("source", **src),
        component("phantom", pos=(0, 0, 0.5), rot=rot_y(angle) if angle else None,
                  nx=n, ny=n, nz=n, voxel=voxel),
        component("mon_epsd", pos=(0, 0, 1.0), nx=n_pix, ny=n_pix, ne=ne,
                  xmin=-half, xmax=half, ymin=-half, ymax=half,
                  e_min=20.0, e_max=160.0),
    ]
    mats = tabulate_materials(PHANTOM_MATERIALS, 20.0, 160.0, 1400)
    if phantom is None:
        phantom = make_phantom(n, seed=phantom_seed)
    return Instrument(components=comps, materials=mats, phantom=phantom,
                      instr_id=instr_id, name=f"ct_{n}cube_{n_pix}x{n_pix}x{ne}",
                      meta={"angle": angle, "window": window})


def rot_x(phi: float) -> tuple:
    """Row-major rotation whose local z axis points along (0, sin phi, cos phi)
    (a turn by -phi about the x axis)."""
    c, s = math.cos(phi), math.sin(phi)
    return (1.0, 0.0, 0.0, 0.0, c, s, 0.0, -s, c)


def edxct_instrument(nx: int = 100, ny: int = 350, nz: int = 250, voxel: float = 1 * MM,
                     n_det: int = 5, det_px: int = 128, pix: float = 0.8 * MM, ne: int = 128,
                     det_dist: float = 2.5, phantom_z: float = 1.5, spot: float = 10e-6,
                     phantom: np.ndarray | None = None, instr_id: int = 0,
                     phantom_x: float = 0.0, phantom_y: float = 0.0,
                     materials: list | None = None) -> Instrument:
    """The paper's energy-dispersive CT line scanner (Sec. 3.3, its table of
    component settings): a 10 x 10 um focal spot with a 160 kV bremsstrahlung
    (Kramers) spectrum, 20-160 keV, as a fan beam onto n_det line detectors of
    1 x det_px pixels (pix square) and ne energy bins, tilted to face the
    source and tiling an arc det_dist from it; in between, a block of water
    voxels, nx (across the fan) x ny (along it) x nz (along the beam), of
    `voxel` edge, centred phantom_z from the source.  The detectors restore
    the ray (each sees every ray of the fan, whatever the order).  The block
    may be moved across the fan (phantom_x: one scan line per position) and
    along it (phantom_y), and its materials replaced (`materials`, material 0
    should stay vacuum)."""
    half_det = 0.5 * det_px * pix
    delta = math.atan(half_det / det_dist)          # half the angle one detector spans
    fan_half = n_det * delta
    comps = [component("source", shape="rect", spot_w=spot, spot_h=spot, spectrum="kramers",
                       e_min=20.0, e_max=160.0, e0=160.0, target_dist=det_dist,
                       target_w=pix, target_h=2 * det_dist * math.tan(fan_half)),
             component("phantom", pos=(phantom_x, phantom_y, phantom_z), nx=nx, ny=ny, nz=nz, voxel=voxel)]
    for k in range(n_det):
        phi = (k - 0.5 * (n_det - 1)) * 2 * delta
        comps.append(component("mon_epsd", pos=(0.0, det_dist * math.sin(phi), det_dist * math.cos(phi)),
                               rot=rot_x(phi), nx=1, ny=det_px, ne=ne,
                               xmin=-0.5 * pix, xmax=0.5 * pix, ymin=-half_det, ymax=half_det,
                               e_min=20.0, e_max=160.0, restore=True))
    mats = tabulate_materials(materials or PHANTOM_MATERIALS[:2], 20.0, 160.0, 1400)
    if phantom is None:
        phantom = np.ones((nz, ny, nx), dtype=np.uint8)   # water everywhere
    return Instrument(components=comps, materials=mats, phantom=phantom, instr_id=instr_id,
                      name=f"edxct_{nx}x{ny}x{nz}_{n_det}x{det_px}x{ne}",
                      meta={"det_dist": det_dist, "delta": delta})


# ---------------------------------------------------------------- staircase test piece
# Synthetic iron and lead for the paper's aviation-security test piece
# (Sec. 5.1): a E^-3 (x5 above lead's K-edge at 88 keV) + b in 1/m, giving
# iron ~15 /cm at 50 keV and ~2.9 /cm at 100 keV, lead ~27 /cm just below its
# K-edge and ~63 /cm at 100 keV.
IRON = (1.728e8, 117.0, None, 1.0)
LEAD = (1.18e9, 395.0, 88.0, 5.0)
STAIRCASE_MATERIALS = [(0.0, 0.0, None, 1.0), IRON, LEAD]

STAIR_STEP_W = 20 * MM       # width of a step along the fan
STAIR_T0, STAIR_DT = 14 * MM, 2 * MM
STAIR_N = 10
STAIR_WIDTH = 60 * MM        # extent across the fan (the scan axis)
STAIR_ROD_R = 5 * MM


def staircase_phantom(voxel: float = 1 * MM) -> np.ndarray:
    """A steel staircase of STAIR_N steps, 14 to 32 mm thick in 2 mm steps
    along the beam (z), each STAIR_STEP_W wide along the fan (y) and
    STAIR_WIDTH across it (x), with a lead rod of radius STAIR_ROD_R along y
    beneath it, centred in x.  Materials: 0 vacuum, 1 iron, 2 lead.  Returned
    as [nz, ny, nx] (x fastest); sizes are whole voxels of `voxel`."""
    v = voxel
    nx = int(round(STAIR_WIDTH / v))
    ny = int(round(STAIR_N * STAIR_STEP_W / v))
    t_max = STAIR_T0 + (STAIR_N - 1) * STAIR_DT
    rod_z0 = int(round((t_max + 1 * MM) / v))          # 1 mm below the thickest step
    nr = int(round(STAIR_ROD_R / v))
    nz = rod_z0 + 2 * nr + 1
    vox = np.zeros((nz, ny, nx), dtype=np.uint8)
    sw = int(round(STAIR_STEP_W / v))
    for k in range(STAIR_N):
        t = int(round((STAIR_T0 + k * STAIR_DT) / v))
        vox[:t, k * sw:(k + 1) * sw, :] = 1
    zc = rod_z0 + nr                                  # rod axis, voxel units
    xc = 0.5 * nx
    z = np.arange(nz)[:, None] + 0.5
    x = np.arange(nx)[None, :] + 0.5
    rod = (z - zc) ** 2 + (x - xc) ** 2 <= nr * nr
    vox[np.broadcast_to(rod[:, None, :], vox.shape)] = 2
    return vox


def staircase_step_y(k: int, voxel: float = 1 * MM) -> float:
    """Local y (phantom frame, grid centred) of the centre of step k."""
    ny = int(round(STAIR_N * STAIR_STEP_W / voxel))
    return (k + 0.5) * STAIR_STEP_W - 0.5 * ny * voxel


def staircase_line(x_line: float, step: int = 6, instr_id: int = 0, voxel: float = 1 * MM,
                   det_px: int = 128, ne: int = 128, phantom: np.ndarray | None = None,
                   n_det: int = 5) -> Instrument:
    """One scan line of the staircase in the EDXCT scanner: the fan crosses
    the phantom at local x = x_line, and step `step` (26 mm for step 6) is
    centred on the central detector."""
    ph = staircase_phantom(voxel) if phantom is None else phantom
    nz, ny, nx = ph.shape
    spec = edxct_instrument(nx=nx, ny=ny, nz=nz, voxel=voxel, n_det=n_det, det_px=det_px, ne=ne, phantom=ph,
                            instr_id=instr_id, phantom_x=-x_line,
                            phantom_y=-staircase_step_y(step, voxel),
                            materials=STAIRCASE_MATERIALS)
    spec.name = f"staircase_line_{x_line * 1e3:+.1f}mm"
    return spec


def staircase_scan(n_lines: int = 10, spacing: float = 1 * MM, **kw):
    """The CNR study's lines (Sec. 5.1): n_lines through the lead rod
    ("ref": steel over lead), n_lines through steel alone ("mat"), and a
    flat-field line that misses the test piece.  Returns (specs, labels)."""
    ref = [(-0.5 * (n_lines - 1) + i) * spacing for i in range(n_lines)]
    mat = [STAIR_ROD_R + 1 * MM + (i + 0.5) * spacing for i in range(n_lines)]
    xs = ref + mat + [10 * STAIR_WIDTH]
    labels = ["ref"] * n_lines + ["mat"] * n_lines + ["flat"]
    specs = [staircase_line(x, instr_id=i, **kw) for i, x in enumerate(xs)]
    return specs, labels


# ---------------------------------------------------------------- focusing instrument
# Synthetic beryllium for the lenses: ~1.2 /cm at 10 keV and ~0.31 /cm at
# 23 keV; refractive decrement 6.26e-7 at 23.32 keV (from the free-electron
# density of Be, 1.85 g/cm^3), scaling as E^-2.
BERYLLIUM = (9.7e4, 23.0, None, 1.0)
BE_DELTA_23 = 6.26e-7


def focusing_instrument(n_lenses: int = 16, radius: float = 200e-6, thickness: float = 50e-6,
                        aperture: float = 0.5 * MM, lens_dist: float = 31.5, slit_dist: float = 14.0,
                        slit_d: float = 0.1 * MM, psd_n: int = 100, psd_w: float = 0.2 * MM,
                        ne: int = 200, delta0: float = BE_DELTA_23, instr_id: int = 0) -> Instrument:
    """The paper's focusing instrument (Sec. 3.2 and its source table): an
    undulator-like Gaussian source (sigma 48.2 x 9.5 um, divergence 100 x 4.3
    urad, E0 = 23.32 keV, sigma_E = 1 keV) aimed at a 1 x 1 mm window at the
    lens centre 31.5 m away; a stack of 16 parabolic Be lenses (R = 200 um,
    apex thickness 50 um, aperture radius 0.5 mm, lenses back to back); a
    circular slit of 0.1 mm diameter 14 m after the lens centre; a PSD and an
    energy monitor just behind it."""
    e0, se = 23.32, 1.0
    src = component("source", shape="gauss", sigma_x=48.2e-6, sigma_y=9.5e-6, div_x=100e-6,
                    div_y=4.3e-6, spectrum="gauss", e0=e0, sigma_e=se, e_min=e0 - 5 * se,
                    e_max=e0 + 5 * se, target_dist=lens_dist, target_w=1 * MM, target_h=1 * MM)
    lens = component("lens_parab", pos=(0, 0, lens_dist), radius=radius, thickness=thickness,
                     aperture=aperture, n_lenses=n_lenses, delta0=delta0, e_ref=e0,
                     pitch=thickness + aperture * aperture / radius, material=0)
    z = lens_dist + slit_dist
    slit = component("slit_circ", pos=(0, 0, z), radius=0.5 * slit_d)
    h = 0.5 * psd_w
    psd = component("mon_psd", pos=(0, 0, z + 1e-3), nx=psd_n, ny=psd_n, xmin=-h, xmax=h, ymin=-h, ymax=h)
    emon = component("mon_e", pos=(0, 0, z + 2e-3), ne=ne, e_min=e0 - 5 * se, e_max=e0 + 5 * se,
                     xmin=-h, xmax=h, ymin=-h, ymax=h)
    mats = tabulate_materials([BERYLLIUM], 10.0, 40.0, 600)
    return Instrument(components=[src, lens, slit, psd, emon], materials=mats, instr_id=instr_id,
                      name=f"focusing_crl{n_lenses}",
                      meta={"focal_length": radius / (2 * n_lenses * delta0) if delta0 > 0 else math.inf})


# ---------------------------------------------------------------- scattering phantom
def edxct_scatter_instrument(**kw) -> Instrument:
    """The EDXCT scanner (edxct_instrument(**kw)) with its block made a
    scatterer, as the paper's phantom is (Sec. 3.3): water's energy-dependent
    Rayleigh and Compton tables (water_scattering) on the 1/3-voxel march."""
    spec = edxct_instrument(**kw)
    spec.components[1]["march"] = 3
    spec.components[1]["scatter"] = True
    m = spec.materials
    spec.mu_scatter, spec.mu_compton = water_scattering((0.0,) + (1.0,) * (m.n_mat - 1), m.e_min,
                                                        m.e_max, m.n_cell)
    return spec


def scatter_block(nx: int = 20, ny: int = 20, nz: int = 20, voxel: float = 2 * MM, s: float = 3.0,
                  mu_s: float = 20.0, absorb: bool = True, seed: int = 7, det_w: float = 0.2,
                  det_n: int = 64, instr_id: int = 0, compton: float = 0.0,
                  energy_dependent: bool = False) -> Instrument:
    """A pencil-like beam (point source, 2 x 2 mm window at 1 m) into a block
    of water-like voxels with random inclusions (seed) that scatters
    (Rayleigh with mu_s per material, 1/m, and Compton with `compton` x
    mu_s) on the fixed-step march at s steps per voxel; a large PSD behind
    the block (det_w square, det_n bins) sees both the direct and the
    scattered rays.  absorb=False keeps scattering only (the attenuation
    tables zero).  energy_dependent: those are the values at 40 keV of
    per-cell tables, Rayleigh falling as E^-2 and Compton following the
    Klein-Nishina cross-section."""
    rng = np.random.default_rng(seed)
    vox = np.ones((nz, ny, nx), dtype=np.uint8)
    vox[rng.random((nz, ny, nx)) < 0.2] = 2
    params = [(0.0, 0.0, None, 1.0), (WATER_A, WATER_B, None, 1.0), (2.0 * WATER_A, 1.2 * WATER_B, None, 1.0)]
    if not absorb:
        params = [(0.0, 0.0, None, 1.0)] * 3
    mats = tabulate_materials(params, 20.0, 120.0, 500)
    comps = [component("source", shape="point", spectrum="flat", e_min=30.0, e_max=90.0,
                       target_dist=1.0, target_w=2 * MM, target_h=2 * MM),
             component("phantom", pos=(0, 0, 1.0), nx=nx, ny=ny, nz=nz, voxel=voxel, march=s,
                       scatter=True),
             component("mon_psd", pos=(0, 0, 1.0 + 0.5 * nz * voxel + 0.05), nx=det_n, ny=det_n,
                       xmin=-0.5 * det_w, xmax=0.5 * det_w, ymin=-0.5 * det_w, ymax=0.5 * det_w)]
    mus = np.array([0.0, mu_s, 2.0 * mu_s])
    muc = compton * mus if compton else None
    if energy_dependent:
        kn40 = klein_nishina_sigma(40.0)
        mus = tabulate_curves([lambda e, v=v: v * (40.0 / e) ** 2 for v in mus], 20.0, 120.0, 500)
        if compton:
            muc = tabulate_curves([lambda e, v=v: v * compton * klein_nishina_sigma(e) / kn40
                                   for v in (0.0, mu_s, 2.0 * mu_s)], 20.0, 120.0, 500)
    return Instrument(components=comps, materials=mats, phantom=vox, instr_id=instr_id,
                      mu_scatter=mus, mu_compton=muc, name="scatter_block")


def batched_workload(n_angles: int = 360, n_slits: int = 16, seed: int = 5,
                     budget_lo: float = 1e6, budget_hi: float = 1e8):
    """Many instruments with uneven ray budgets: `n_angles` projections of the
    absorption instrument (cylinder rotated about its axis, budgets
    log-uniform in [budget_lo, budget_hi]) plus `n_slits` flat-slit
    instruments with slit widths log-spaced over 0.1-2 mm (1e6 rays each).
    Returns (instruments, budgets)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    budgets = np.exp(rng.uniform(math.log(budget_lo), math.log(budget_hi), size=n_angles))
    budgets = np.sort(budgets.astype(np.int64))[::-1]
    insts, buds = [], []
    for i in range(n_angles):
        insts.append(absorption_instrument(angle=2 * math.pi * i / max(n_angles, 1),
                                           instr_id=i))
        buds.append(int(budgets[i]))
    widths = np.exp(np.linspace(math.log(0.1 * MM), math.log(2.0 * MM), n_slits)) if n_slits else []
    for j, w in enumerate(widths):
        insts.append(flat_slit_instrument(slit_w=float(w), instr_id=n_angles + j))
        buds.append(1_000_000)
    return insts, buds


# ---------------------------------------------------------------- learned proposal
PROPOSAL_HIDDEN = 128
PROPOSAL_COMPONENTS = 8


def proposal_init(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters of the direction proposal network, flat in the
    order W1 [4,128], b1, W2 [128,128], b2, W3 [128,128], b3, W4 [128,40], b4:
    normal weights scaled by 1/sqrt(fan-in), zero biases, the last layer's
    weights shrunk by 10 and its bias set to a broad mixture (components on a
    ring of radius 0.5, log-width outputs 1).  Output layout per component:
    (logit, mu_u, mu_v, width_u, width_v)."""
    h, k = PROPOSAL_HIDDEN, PROPOSAL_COMPONENTS
    rng = np.random.Generator(np.random.PCG64(seed))
    shapes = [(4, h), (h,), (h, h), (h,), (h, h), (h,), (h, 5 * k), (5 * k,)]
    ps = []
    for s in shapes:
        ps.append(rng.normal(0.0, 1.0 / math.sqrt(s[0]), size=s) if len(s) == 2 else np.zeros(s))
    ps[6] *= 0.1
    b4 = ps[7].reshape(k, 5)
    ang = 2 * np.pi * np.arange(k) / k
    b4[:, 1] = 0.5 * np.cos(ang)
    b4[:, 2] = 0.5 * np.sin(ang)
    b4[:, 3] = 1.0
    b4[:, 4] = 1.0
    return np.concatenate([p.ravel() for p in ps])
