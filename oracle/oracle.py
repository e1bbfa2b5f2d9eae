"""CPU oracle of the forward Monte Carlo X-ray ray tracer (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module.  It never imports the
GPU package: it takes instrument descriptions as plain data (objects with
``components``, ``materials``, ``phantom`` and ``instr_id`` attributes) and
marshals them with its own code into the C oracle's structs (``orc.h``).

The C sources are plain binary64 per-ray loops (``orc_core.inc``); this file
only places components in the lab frame (x_lab = o + R x_local, composed
along ``relative_to``), lays the monitor bins end to end, and optionally
splits a ray range over host threads with private monitors that are summed
afterwards (the scatter/gather of the paper's MPI mode, Sec. 2.2.1).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ("orc_rng.c", "orc_geom.c", "orc_trace.c")
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lib = None
_lock = threading.Lock()

TYPE_CODES = {
    "source": 0, "slit_rect": 1, "slit_circ": 2, "abs_box": 3, "abs_cyl": 4,
    "abs_sphere": 5, "phantom": 6, "mon_psd": 7, "mon_e": 8, "mon_l": 9,
    "mon_epsd": 10, "lens_parab": 11,
}
SHAPES = {"point": 0, "disk": 1, "rect": 2, "gauss": 3}
SPECTRA = {"flat": 0, "kramers": 1, "gauss": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    deps = srcs + [os.path.join(_HERE, "orc.h"), os.path.join(_HERE, "orc_core.inc")]
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(d) for d in deps)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcComp(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("shape", ctypes.c_int32),
                ("spectrum", ctypes.c_int32), ("material", ctypes.c_int32),
                ("n", ctypes.c_int32 * 3), ("pad", ctypes.c_int32),
                ("mon_offset", ctypes.c_int64), ("o", ctypes.c_double * 3),
                ("R", ctypes.c_double * 9), ("a", ctypes.c_double * 12)]


class OrcInstrument(ctypes.Structure):
    _fields_ = [("n_comp", ctypes.c_int32), ("n_mat", ctypes.c_int32),
                ("n_cell", ctypes.c_int32), ("instr_id", ctypes.c_int32),
                ("comp", ctypes.POINTER(OrcComp)), ("e_min", ctypes.c_double),
                ("e_max", ctypes.c_double), ("coef", ctypes.POINTER(ctypes.c_double)),
                ("vox", ctypes.POINTER(ctypes.c_uint8)),
                ("mus", ctypes.POINTER(ctypes.c_double)),
                ("muc", ctypes.POINTER(ctypes.c_double))]


class OrcOut(ctypes.Structure):
    _fields_ = [("N", ctypes.POINTER(ctypes.c_int64)), ("sw", ctypes.POINTER(ctypes.c_double)),
                ("sw2", ctypes.POINTER(ctypes.c_double)), ("lost", ctypes.POINTER(ctypes.c_double)),
                ("n_emit", ctypes.c_int64), ("sum_w0", ctypes.c_double),
                ("sum_wend", ctypes.c_double)]


def _configure(L):
    """Declare the C oracle's signatures on a loaded library."""
    d3 = ctypes.POINTER(ctypes.c_double)
    L.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
    L.orc_uniform64.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
    L.orc_uniform64.restype = ctypes.c_double
    L.orc_uniform32.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
    L.orc_uniform32.restype = ctypes.c_float
    L.orc_chord_box.argtypes = [d3, d3, d3]
    L.orc_chord_box.restype = ctypes.c_double
    L.orc_chord_cyl.argtypes = [d3, d3, ctypes.c_double, ctypes.c_double]
    L.orc_chord_cyl.restype = ctypes.c_double
    L.orc_chord_sphere.argtypes = [d3, d3, ctypes.c_double]
    L.orc_chord_sphere.restype = ctypes.c_double
    L.orc_siddon_tau.argtypes = [d3, d3, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.POINTER(ctypes.c_uint8), d3]
    L.orc_siddon_tau.restype = ctypes.c_double
    L.orc_march_tau.argtypes = [d3, d3, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.c_double, ctypes.POINTER(ctypes.c_uint8), d3]
    L.orc_march_tau.restype = ctypes.c_double
    L.orc_ln64.argtypes = [ctypes.c_double]
    L.orc_ln64.restype = ctypes.c_double
    L.orc_ln32.argtypes = [ctypes.c_float]
    L.orc_ln32.restype = ctypes.c_float
    L.orc_lens_ray.argtypes = [ctypes.c_void_p, d3, d3, ctypes.c_double, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_double)]
    L.orc_lens_ray.restype = ctypes.c_int
    L.orc_scatter_dir.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_double, d3,
                                  ctypes.POINTER(ctypes.c_double)]
    L.orc_scatter_dir.restype = ctypes.c_uint32
    L.orc_aim_direction.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), d3]
    L.orc_aim_direction.restype = None
    L.orc_mu.argtypes = [ctypes.POINTER(OrcInstrument), ctypes.c_int, ctypes.c_double, ctypes.c_int]
    L.orc_mu.restype = ctypes.c_double
    L.orc_trace.argtypes = [ctypes.POINTER(OrcInstrument), ctypes.c_uint64, ctypes.c_uint64,
                            ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(OrcOut)]
    L.orc_trace.restype = ctypes.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(ctypes.CDLL(_LIB_PATH))
    return _lib


def build_variant(patches, directory: str):
    """Compile a deliberately altered copy of the oracle into `directory` and
    load it.  `patches` is a list of (file, old, new) text replacements, each
    of which must match exactly once.  Tests use this to plant a mistake in
    the oracle and show that a pin catches it; nothing else may."""
    os.makedirs(directory, exist_ok=True)
    texts = {}
    for name in _SOURCES + ("orc.h", "orc_core.inc"):
        with open(os.path.join(_HERE, name)) as f:
            texts[name] = f.read()
    for name, old, new in patches:
        if texts[name].count(old) != 1:
            raise ValueError(f"patch target not found exactly once in {name}: {old!r}")
        texts[name] = texts[name].replace(old, new)
    for name, text in texts.items():
        with open(os.path.join(directory, name), "w") as f:
            f.write(text)
    path = os.path.join(directory, "liborc_variant.so")
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", path] + [os.path.join(directory, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    return _configure(ctypes.CDLL(path))


# ------------------------------------------------------------------ primitives
def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform64(ray_id: int, instr: int, seed: int, j: int) -> float:
    return lib().orc_uniform64(ray_id, instr, seed, j)


def uniform32(ray_id: int, instr: int, seed: int, j: int) -> float:
    return lib().orc_uniform32(ray_id, instr, seed, j)


def aim_direction(mode: int, sx: float, sy: float, tx: float, ty: float, tz: float, lib_=None):
    """Unit direction from (sx, sy, 0) towards (tx, ty, tz) as the ray loop
    forms it (mode 64 binary64, mode 32 binary32)."""
    L = lib_ or lib()
    a = (ctypes.c_double * 5)(sx, sy, tx, ty, tz)
    k = (ctypes.c_double * 3)()
    L.orc_aim_direction(mode, a, k)
    return [k[0], k[1], k[2]]


def _d3(v):
    return (ctypes.c_double * 3)(*[float(a) for a in v])


def chord_box(x, k, w):
    return lib().orc_chord_box(_d3(x), _d3(k), _d3(w))


def chord_cyl(x, k, radius, height):
    return lib().orc_chord_cyl(_d3(x), _d3(k), float(radius), float(height))


def chord_sphere(x, k, radius):
    return lib().orc_chord_sphere(_d3(x), _d3(k), float(radius))


def siddon_tau(x, k, vox: np.ndarray, voxel: float, mu_mat) -> float:
    """Line integral of mu over a centred voxel grid ``vox[nz, ny, nx]``."""
    vox = np.ascontiguousarray(vox, dtype=np.uint8)
    mu = np.ascontiguousarray(mu_mat, dtype=np.float64)
    nz, ny, nx = vox.shape
    return lib().orc_siddon_tau(_d3(x), _d3(k), nx, ny, nz, float(voxel),
                                vox.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))


def march_tau(x, k, vox: np.ndarray, voxel: float, steps_per_voxel: float, mu_mat) -> float:
    """The fixed-step traversal of the same grid (Sec. 3.3): steps of
    voxel / steps_per_voxel, each weighted by the voxel at its end point."""
    vox = np.ascontiguousarray(vox, dtype=np.uint8)
    mu = np.ascontiguousarray(mu_mat, dtype=np.float64)
    nz, ny, nx = vox.shape
    return lib().orc_march_tau(_d3(x), _d3(k), nx, ny, nz, float(voxel), float(voxel) / float(steps_per_voxel),
                               vox.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                               mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))


def ln64(x: float) -> float:
    """The contract's logarithm in binary64 (orc.h)."""
    return lib().orc_ln64(float(x))


def ln32(x) -> float:
    """The contract's logarithm in binary32."""
    return lib().orc_ln32(float(np.float32(x)))


def scatter_dir(ray_id: int, instr: int, seed: int, j: int, mr: float, mc: float, k, E: float,
                mode: int = 64):
    """One scattering event of the phantom's sampler from draw j on, for a
    material with Rayleigh and Compton coefficients mr, mc: (new k, new E, next j)."""
    ka = _d3(k)
    e = ctypes.c_double(float(E))
    nj = lib().orc_scatter_dir(int(ray_id), int(instr), int(seed), int(j), int(mode), float(mr), float(mc),
                               ka, ctypes.byref(e))
    return np.array(list(ka)), e.value, int(nj)


def lens_ray(comp: dict, x, k, E: float, mode: int = 64):
    """One ray through a lens_parab component dict in its local frame:
    returns (passed, x, k, path length in the lens material)."""
    oc = OrcComp()
    oc.type = TYPE_CODES["lens_parab"]
    oc.a[:7] = [comp["radius"], comp["thickness"], comp["aperture"], float(comp["n_lenses"]),
                comp["delta0"], comp["e_ref"], comp["pitch"]]
    oc.n[:] = [int(comp["n_lenses"]), 1, 1]
    xa, ka = _d3(x), _d3(k)
    path = ctypes.c_double(0.0)
    ok = lib().orc_lens_ray(ctypes.addressof(oc), xa, ka, float(E), int(mode), ctypes.byref(path))
    if ok < 0:
        raise ValueError("not a lens")
    return bool(ok), np.array(list(xa)), np.array(list(ka)), path.value


# ------------------------------------------------------------------ instruments
def _rot(r):
    return np.eye(3) if r is None else np.asarray(r, dtype=np.float64).reshape(3, 3)


def place(components):
    """Lab-frame (origin, rotation) of every component: a component placed
    `relative_to` p sits at o_p + R_p pos with rotation R_p rot.  Sums are
    taken left to right, one rounding per operation."""
    frames = []
    for i, c in enumerate(components):
        pos = [float(v) for v in c["pos"]]
        rot = _rot(c.get("rot")).reshape(-1).tolist()
        p = c.get("relative_to", -1)
        if p is None or p < 0:
            frames.append((np.array(pos), np.array(rot).reshape(3, 3)))
            continue
        if p >= i:
            raise ValueError("relative_to must name an earlier component")
        op, Rp = frames[p]
        Rq = Rp.reshape(-1).tolist()
        o = [float(op[r]) + ((Rq[3 * r] * pos[0] + Rq[3 * r + 1] * pos[1]) + Rq[3 * r + 2] * pos[2])
             for r in range(3)]
        R = [(Rq[3 * r] * rot[col] + Rq[3 * r + 1] * rot[3 + col]) + Rq[3 * r + 2] * rot[6 + col]
             for r in range(3) for col in range(3)]
        frames.append((np.array(o), np.array(R).reshape(3, 3)))
    return frames


def _monitor_bins(c):
    t = c["type"]
    return {"mon_psd": lambda: c["nx"] * c["ny"], "mon_e": lambda: c["ne"],
            "mon_l": lambda: c["nl"], "mon_epsd": lambda: c["nx"] * c["ny"] * c["ne"]
            }.get(t, lambda: 0)()


class Compiled:
    """An instrument marshalled into the oracle's C structs."""

    def __init__(self, inst):
        comps = inst.components
        frames = place(comps)
        self.n_comp = len(comps)
        self.comp = (OrcComp * self.n_comp)()
        self.mon_slices = {}
        off = 0
        for i, (c, (o, R)) in enumerate(zip(comps, frames)):
            oc = self.comp[i]
            oc.type = TYPE_CODES[c["type"]]
            oc.material = int(c.get("material", 0))
            oc.o[:] = [float(v) for v in o]
            oc.R[:] = [float(v) for v in R.reshape(-1)]
            a = [0.0] * 12
            n = [1, 1, 1]
            t = c["type"]
            if t == "source":
                oc.shape = SHAPES[c["shape"]]
                oc.spectrum = SPECTRA[c["spectrum"]]
                if c["shape"] == "disk":
                    a[0] = c["radius"]
                elif c["shape"] == "rect":
                    a[0], a[1] = c["spot_w"], c["spot_h"]
                elif c["shape"] == "gauss":
                    a[0], a[1] = c["sigma_x"], c["sigma_y"]
                    a[9], a[10] = c.get("div_x", 0.0), c.get("div_y", 0.0)
                a[2], a[3] = c["e_min"], c["e_max"]
                a[4] = c.get("e0", c["e_max"])
                a[8] = c.get("sigma_e", 0.0)
                a[5], a[6], a[7] = c["target_dist"], c["target_w"], c["target_h"]
            elif t == "slit_rect":
                a[:4] = [c["xmin"], c["xmax"], c["ymin"], c["ymax"]]
            elif t == "slit_circ":
                a[0] = c["radius"]
            elif t == "abs_box":
                a[:3] = [c["wx"], c["wy"], c["wz"]]
            elif t == "abs_cyl":
                a[:2] = [c["radius"], c["height"]]
            elif t == "abs_sphere":
                a[0] = c["radius"]
            elif t == "phantom":
                a[0] = c["voxel"]
                a[1] = float(c.get("march", 0))
                a[4] = 1.0 if c.get("scatter") else 0.0
                n = [c["nx"], c["ny"], c["nz"]]
            elif t == "lens_parab":
                a[:7] = [c["radius"], c["thickness"], c["aperture"], float(c["n_lenses"]),
                         c["delta0"], c["e_ref"], c["pitch"]]
                n = [int(c["n_lenses"]), 1, 1]
            elif t in ("mon_psd", "mon_e", "mon_l", "mon_epsd"):
                a[:4] = [c["xmin"], c["xmax"], c["ymin"], c["ymax"]]
                if t == "mon_psd":
                    n = [c["nx"], c["ny"], 1]
                elif t == "mon_e":
                    a[4], a[5] = c["e_min"], c["e_max"]
                    n = [c["ne"], 1, 1]
                elif t == "mon_l":
                    a[4], a[5] = c["l_min"], c["l_max"]
                    n = [c["nl"], 1, 1]
                else:
                    a[4], a[5] = c["e_min"], c["e_max"]
                    n = [c["nx"], c["ny"], c["ne"]]
                a[11] = 1.0 if c.get("restore") else 0.0
                nb = _monitor_bins(c)
                oc.mon_offset = off
                self.mon_slices[i] = (off, nb)
                off += nb
            oc.a[:] = [float(v) for v in a]
            oc.n[:] = n
        self.n_bins = off
        self.ins = OrcInstrument()
        self.ins.n_comp = self.n_comp
        self.ins.comp = ctypes.cast(self.comp, ctypes.POINTER(OrcComp))
        self.ins.instr_id = int(inst.instr_id)
        mats = inst.materials
        if mats is not None:
            self.coef = np.ascontiguousarray(mats.coef, dtype=np.float64)
            self.ins.n_mat, self.ins.n_cell = self.coef.shape[0], self.coef.shape[1]
            self.ins.e_min, self.ins.e_max = float(mats.e_min), float(mats.e_max)
            self.ins.coef = self.coef.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if inst.phantom is not None:
            ph = [c for c in comps if c["type"] == "phantom"][0]
            self.vox = np.ascontiguousarray(inst.phantom, dtype=np.uint8)
            if self.vox.shape != (ph["nz"], ph["ny"], ph["nx"]):
                raise ValueError("phantom bytes do not match the phantom component")
            self.ins.vox = self.vox.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        if getattr(inst, "mu_scatter", None) is not None:
            self.mus = self._scatter_table(inst.mu_scatter)
            self.ins.mus = self.mus.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if getattr(inst, "mu_compton", None) is not None:
            self.muc = self._scatter_table(inst.mu_compton)
            self.ins.muc = self.muc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def _scatter_table(self, a):
        """A scattering coefficient as the oracle's per-cell table
        [n_mat][n_cell][2]: given as that table, or one energy-independent
        value per material (the table with zero slopes)."""
        a = np.asarray(a, dtype=np.float64)
        nm, nc = self.ins.n_mat, self.ins.n_cell
        if a.shape == (nm,):
            t = np.zeros((nm, nc, 2))
            t[:, :, 0] = a[:, None]
            return t
        if a.shape != (nm, nc, 2):
            raise ValueError("scattering coefficients: one per material or a (n_mat, n_cell, 2) table")
        return np.ascontiguousarray(a)


class Result:
    """Monitor sums and loss tallies of an oracle run."""

    def __init__(self, compiled: Compiled):
        n = max(compiled.n_bins, 1)
        self.N = np.zeros(n, dtype=np.int64)
        self.sw = np.zeros(n, dtype=np.float64)
        self.sw2 = np.zeros(n, dtype=np.float64)
        self.lost = np.zeros(compiled.n_comp, dtype=np.float64)
        self.n_emit = 0
        self.sum_w0 = 0.0
        self.sum_wend = 0.0
        self._slices = compiled.mon_slices

    def monitor(self, comp_index: int):
        off, nb = self._slices[comp_index]
        return self.N[off:off + nb], self.sw[off:off + nb], self.sw2[off:off + nb]

    def add(self, other: "Result"):
        self.N += other.N
        self.sw += other.sw
        self.sw2 += other.sw2
        self.lost += other.lost
        self.n_emit += other.n_emit
        self.sum_w0 += other.sum_w0
        self.sum_wend += other.sum_wend


def _run(compiled: Compiled, begin: int, end: int, seed: int, mode: int, res: Result, L=None):
    out = OrcOut()
    out.N = res.N.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    out.sw = res.sw.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    out.sw2 = res.sw2.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    out.lost = res.lost.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = (L or lib()).orc_trace(ctypes.byref(compiled.ins), begin, end, seed, mode, ctypes.byref(out))
    if rc != 0:
        raise ValueError("oracle rejected the instrument")
    res.n_emit += out.n_emit
    res.sum_w0 += out.sum_w0
    res.sum_wend += out.sum_wend


def trace(inst, ray_begin: int, ray_end: int, seed: int, mode: int = 64,
          threads: int = 1, compiled: Compiled | None = None, lib_=None) -> Result:
    """Trace rays [ray_begin, ray_end) of `inst` under `seed`.

    mode 64 is the all-binary64 reference; mode 32 takes the sampled ray and
    every count-deciding quantity in binary32, as the mixed-precision GPU
    path does, with weights in binary64.  With threads > 1 the range is cut
    into contiguous pieces traced concurrently into private results that are
    then summed (ctypes releases the GIL during each call).  `lib_` selects
    a library from build_variant instead of the oracle itself."""
    comp = compiled if compiled is not None else Compiled(inst)
    total = Result(comp)
    n = ray_end - ray_begin
    threads = max(1, min(int(threads), max(n, 1)))
    if threads == 1:
        _run(comp, ray_begin, ray_end, seed, mode, total, lib_)
        return total
    cuts = [ray_begin + (n * i) // threads for i in range(threads + 1)]
    parts = [Result(comp) for _ in range(threads)]
    ths = [threading.Thread(target=_run, args=(comp, cuts[i], cuts[i + 1], seed, mode, parts[i], lib_))
           for i in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    for p in parts:
        total.add(p)
    return total


def mu(inst, material: int, E: float, mode: int = 64) -> float:
    comp = Compiled(inst)
    return lib().orc_mu(ctypes.byref(comp.ins), int(material), float(E), int(mode))


def _lib_starts():
    L = lib()
    if not getattr(L, "_starts_ready", False):
        L.orc_sample_starts.argtypes = [ctypes.POINTER(OrcInstrument), ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.POINTER(ctypes.c_float)]
        L.orc_sample_starts.restype = ctypes.c_int
        L.orc_trace_starts.argtypes = [ctypes.POINTER(OrcInstrument), ctypes.POINTER(ctypes.c_float),
                                       ctypes.c_uint64, ctypes.POINTER(OrcOut),
                                       ctypes.POINTER(ctypes.c_double)]
        L.orc_trace_starts.restype = ctypes.c_int
        L._starts_ready = True
    return L


def sample_starts(inst, ray_begin: int, n: int, seed: int) -> np.ndarray:
    """Mode-32 ray starts of rays [ray_begin, ray_begin + n): float32 rows
    (sx, sy, E, u, v, w0), shape (6, n)."""
    comp = Compiled(inst)
    out = np.zeros((6, n), dtype=np.float32)
    rc = _lib_starts().orc_sample_starts(ctypes.byref(comp.ins), ray_begin, n, seed,
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    if rc != 0:
        raise ValueError("oracle rejected the instrument")
    return out


def trace_starts(inst, starts: np.ndarray):
    """Mode-32 trace of given ray starts (6, n); returns (Result, detected
    weight per ray at the last component)."""
    comp = Compiled(inst)
    st = np.ascontiguousarray(starts, dtype=np.float32)
    n = st.shape[1]
    res = Result(comp)
    det = np.zeros(n, dtype=np.float64)
    out = OrcOut()
    out.N = res.N.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    out.sw = res.sw.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    out.sw2 = res.sw2.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    out.lost = res.lost.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = _lib_starts().orc_trace_starts(ctypes.byref(comp.ins),
                                        st.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n,
                                        ctypes.byref(out), det.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("oracle rejected the instrument")
    res.n_emit += out.n_emit
    res.sum_w0 += out.sum_w0
    res.sum_wend += out.sum_wend
    return res, det
