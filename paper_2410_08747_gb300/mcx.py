"""Thin ctypes binding of the C ABI in ``include/mcx.h`` (``libmcx.so``).

Argument marshalling only: every step of a trace runs in the CUDA library.
PyTorch supplies the device memory (through the allocation hook) and the
stream (the current torch stream) when it is available.  There is no CPU
fallback: if the library is missing, every call raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import workloads as wl

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmcx.so")

MCX_OK = 0
STATUS = {0: "MCX_OK", -1: "MCX_ERR_INVALID", -2: "MCX_ERR_OOM", -3: "MCX_ERR_CUDA",
          -4: "MCX_ERR_TIMEOUT", -5: "MCX_ERR_DEVICE", -6: "MCX_ERR_UNSUPPORTED"}
TYPES = {"source": 0, "slit_rect": 1, "slit_circ": 2, "abs_box": 3, "abs_cyl": 4,
         "abs_sphere": 5, "phantom": 6, "mon_psd": 7, "mon_e": 8, "mon_l": 9, "mon_epsd": 10,
         "lens_parab": 11}
SHAPES = {"point": 0, "disk": 1, "rect": 2, "gauss": 3}
SPECTRA = {"flat": 0, "kramers": 1, "gauss": 2}
PRECISIONS = {"fp64": 0, "mixed": 1}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class ComponentDesc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("relative_to", ctypes.c_int32),
                ("shape", ctypes.c_int32), ("spectrum", ctypes.c_int32),
                ("material", ctypes.c_int32), ("n", ctypes.c_int32 * 3),
                ("pos", ctypes.c_double * 3), ("rot", ctypes.c_double * 9),
                ("p", ctypes.c_double * 12)]


class MaterialTables(ctypes.Structure):
    _fields_ = [("n_mat", ctypes.c_int32), ("n_cell", ctypes.c_int32),
                ("e_min", ctypes.c_double), ("e_max", ctypes.c_double),
                ("coef", ctypes.POINTER(ctypes.c_double))]


class Phantom(ctypes.Structure):
    _fields_ = [("vox", ctypes.POINTER(ctypes.c_uint8)), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("mu_scatter", ctypes.POINTER(ctypes.c_double)),
                ("mu_compton", ctypes.POINTER(ctypes.c_double))]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("instr_id", ctypes.c_int32),
                ("device", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("stream", ctypes.c_void_p)]


class BatchOptions(ctypes.Structure):
    _fields_ = [("chunk_rays", ctypes.c_uint64), ("block_size", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class McxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lib_lock = threading.Lock()


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lib_lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.POINTER
            L.mcx_instrument_create.argtypes = [P(ComponentDesc), ctypes.c_int32, P(MaterialTables),
                                                P(Phantom), P(Options), P(ctypes.c_void_p)]
            L.mcx_trace_range.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            L.mcx_trace.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]
            L.mcx_monitor_bins.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_size_t)]
            L.mcx_monitor_read.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
            L.mcx_monitor_read_async.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
            L.mcx_tally_read.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         P(ctypes.c_uint64), P(ctypes.c_double), P(ctypes.c_double)]
            L.mcx_monitor_reset.argtypes = [ctypes.c_void_p]
            L.mcx_synchronize.argtypes = [ctypes.c_void_p]
            L.mcx_instrument_destroy.argtypes = [ctypes.c_void_p]
            L.mcx_instrument_destroy.restype = None
            L.mcx_last_error.restype = ctypes.c_char_p
            L.mcx_philox_fill.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32]
            L.mcx_convert_fill.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_int32]
            L.mcx_batch_create.argtypes = [P(ctypes.c_void_p), P(ctypes.c_uint64), ctypes.c_int32,
                                           P(BatchOptions), P(ctypes.c_void_p)]
            L.mcx_batch_trace.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
            L.mcx_batch_autotune.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                             P(BatchOptions)]
            L.mcx_batch_items.argtypes = [ctypes.c_void_p, P(ctypes.c_uint64)]
            L.mcx_batch_specialize.argtypes = [ctypes.c_void_p, ctypes.c_int32]
            L.mcx_batch_specialize.restype = ctypes.c_int
            L.mcx_batch_destroy.argtypes = [ctypes.c_void_p]
            L.mcx_batch_destroy.restype = None
            L.mcx_batch_trace_static.argtypes = [P(ctypes.c_void_p), P(ctypes.c_uint64), ctypes.c_int32,
                                                 ctypes.c_uint64, ctypes.c_uint64]
            L.mcx_batch_trace_static.restype = ctypes.c_int
            L.mcx_sample_starts.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_uint64, ctypes.c_void_p]
            L.mcx_sample_starts.restype = ctypes.c_int
            L.mcx_trace_starts.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                           ctypes.c_uint64, ctypes.c_void_p]
            L.mcx_trace_starts.restype = ctypes.c_int
            L.mcx_instrument_specialize.argtypes = [ctypes.c_void_p, ctypes.c_int32]
            L.mcx_instrument_specialize.restype = ctypes.c_int
            L.mcx_instrument_source.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t,
                                                P(ctypes.c_size_t)]
            L.mcx_instrument_source.restype = ctypes.c_int
            L.mcx_monitor_total.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_uint64),
                                            P(ctypes.c_double), P(ctypes.c_double)]
            L.mcx_monitor_total.restype = ctypes.c_int
            L.mcx_loss_read.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
            L.mcx_loss_read.restype = ctypes.c_int
            L.mcx_peak_measure.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                           P(ctypes.c_double)]
            L.mcx_peak_measure.restype = ctypes.c_int
            for name in ("mcx_instrument_create", "mcx_trace_range", "mcx_trace", "mcx_monitor_bins",
                         "mcx_monitor_read", "mcx_monitor_read_async", "mcx_tally_read", "mcx_monitor_reset",
                         "mcx_synchronize",
                         "mcx_philox_fill", "mcx_convert_fill", "mcx_batch_create", "mcx_batch_trace",
                         "mcx_batch_autotune", "mcx_batch_items"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def check(status: int):
    if status != MCX_OK:
        raise McxError(status, lib().mcx_last_error().decode())


def philox_fill(ctr_key: np.ndarray, device: int = 0) -> np.ndarray:
    """Device Philox4x32-10 of each row (c0, c1, c2, c3, k0, k1) -> (n, 4) words."""
    a = np.ascontiguousarray(ctr_key, dtype=np.uint32).reshape(-1, 6)
    out = np.zeros((a.shape[0], 4), dtype=np.uint32)
    check(lib().mcx_philox_fill(a.ctypes.data, out.ctypes.data, a.shape[0], int(device)))
    return out


PEAK_KINDS = {"ffma": 0, "imad": 1, "philox": 2, "dfma": 3, "hit": 4, "red_u64": 5}


def peak_measure(kind: str, device: int = 0, footprint_bytes: int = 0) -> float:
    """The library's microbenchmark of one hardware unit (mcx.h, peaks):
    operations per second (FFMA, IMAD, DFMA lane instructions; Philox blocks;
    monitor hits of three atomics; u64 atomic adds)."""
    out = ctypes.c_double(0.0)
    check(lib().mcx_peak_measure(PEAK_KINDS[kind], int(device), int(footprint_bytes), ctypes.byref(out)))
    return out.value


# ------------------------------------------------------------------ marshalling
def scatter_table(a, coef_shape) -> np.ndarray:
    """A scattering coefficient as the library takes it: a per-cell table
    [n_mat][n_cell][2] shaped like the attenuation tables (returned as is),
    or one energy-independent value per material (the table with zero
    slopes)."""
    a = np.asarray(a, dtype=np.float64)
    nm, nc = int(coef_shape[0]), int(coef_shape[1])
    if a.shape == (nm,):
        t = np.zeros((nm, nc, 2))
        t[:, :, 0] = a[:, None]
        return t
    if a.shape != (nm, nc, 2):
        raise ValueError("scattering coefficients: one per material or a (n_mat, n_cell, 2) table")
    return np.ascontiguousarray(a)


def component_desc(c: dict) -> ComponentDesc:
    """One workloads component dict -> mcx_component_desc (see mcx.h for p[])."""
    d = ComponentDesc()
    t = c["type"]
    d.type = TYPES[t]
    d.relative_to = int(c.get("relative_to", -1))
    d.pos[:] = [float(v) for v in c["pos"]]
    rot = c.get("rot")
    d.rot[:] = [1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0] if rot is None else [float(v) for v in rot]
    p = [0.0] * 12
    n = [0, 0, 0]
    if t == "source":
        d.shape = SHAPES[c["shape"]]
        d.spectrum = SPECTRA[c["spectrum"]]
        if c["shape"] == "disk":
            p[0] = c["radius"]
        elif c["shape"] == "rect":
            p[0], p[1] = c["spot_w"], c["spot_h"]
        elif c["shape"] == "gauss":
            p[0], p[1] = c["sigma_x"], c["sigma_y"]
            p[9], p[10] = c.get("div_x", 0.0), c.get("div_y", 0.0)
        p[2], p[3] = c["e_min"], c["e_max"]
        p[4] = c.get("e0", c["e_max"])
        p[8] = c.get("sigma_e", 0.0)
        p[5], p[6], p[7] = c["target_dist"], c["target_w"], c["target_h"]
    elif t == "slit_rect":
        p[:4] = [c["xmin"], c["xmax"], c["ymin"], c["ymax"]]
    elif t == "slit_circ":
        p[0] = c["radius"]
    elif t in ("abs_box", "abs_cyl", "abs_sphere"):
        d.material = int(c["material"])
        if t == "abs_box":
            p[:3] = [c["wx"], c["wy"], c["wz"]]
        elif t == "abs_cyl":
            p[:2] = [c["radius"], c["height"]]
        else:
            p[0] = c["radius"]
    elif t == "phantom":
        p[0] = c["voxel"]
        p[1] = float(c.get("march", 0))
        p[4] = 1.0 if c.get("scatter") else 0.0
        n = [c["nx"], c["ny"], c["nz"]]
    elif t == "lens_parab":
        d.material = int(c["material"])
        p[:7] = [c["radius"], c["thickness"], c["aperture"], float(c["n_lenses"]), c["delta0"],
                 c["e_ref"], c["pitch"]]
        n = [int(c["n_lenses"]), 1, 1]
    else:
        p[:4] = [c["xmin"], c["xmax"], c["ymin"], c["ymax"]]
        if t == "mon_psd":
            n = [c["nx"], c["ny"], 1]
        elif t == "mon_e":
            p[4], p[5] = c["e_min"], c["e_max"]
            n = [c["ne"], 1, 1]
        elif t == "mon_l":
            p[4], p[5] = c["l_min"], c["l_max"]
            n = [c["nl"], 1, 1]
        elif t == "mon_epsd":
            p[4], p[5] = c["e_min"], c["e_max"]
            n = [c["nx"], c["ny"], c["ne"]]
        p[11] = 1.0 if c.get("restore") else 0.0
    d.p[:] = [float(v) for v in p]
    d.n[:] = [int(v) for v in n]
    return d


def convert_fill(values, device: int = 0):
    """Device rounding binary64 -> binary32 and widening back, as the mixed
    form performs them: returns (float32 array, float64 array)."""
    a = np.ascontiguousarray(values, dtype=np.float64).ravel()
    of = np.zeros(a.size, dtype=np.float32)
    od = np.zeros(a.size, dtype=np.float64)
    check(lib().mcx_convert_fill(a.ctypes.data, of.ctypes.data, od.ctypes.data, a.size, int(device)))
    return of, od


def _host_ptr(a, n, dtype):
    """Address of a contiguous host array of n elements of `dtype` (numpy or
    a CPU torch tensor), checked."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype) or a.size != n or not a.flags.c_contiguous:
            raise ValueError(f"need a contiguous {dtype} array of {n} elements")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if str(a.dtype).split(".")[-1] != dtype or a.numel() != n or not a.is_contiguous() \
                or a.device.type != "cpu":
            raise ValueError(f"need a contiguous CPU {dtype} tensor of {n} elements")
        return a.data_ptr()
    raise TypeError("monitor output must be a numpy array or a CPU tensor")


class _TorchAllocator:
    """Device buffers from the PyTorch caching allocator, kept alive by id."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, _ctx):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=f"cuda:{self.device}")
        except Exception:
            return None
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, _ctx):
        self.live.pop(ptr, None)


class Instrument:
    """A traced instrument living on one GPU.

    ``precision`` is "fp64" (plain form) or "mixed" (binary32 propagation,
    binary64 frames and sums).  ``stream`` is a CUDA stream handle (int) or
    None for the current torch stream.  Device memory comes from the torch
    caching allocator, or from ``allocator`` (an object with ``alloc_cb`` and
    ``free_cb`` ctypes callbacks) when given, or from cudaMalloc when
    ``torch_alloc`` is False."""

    def __init__(self, inst: wl.Instrument, precision: str = "fp64", device: int = 0,
                 stream=None, block_size: int = 0, blocks_per_sm: int = 0,
                 torch_alloc: bool = True, allocator=None, specialize: bool = False):
        L = lib()
        self.spec = inst
        comps = inst.components
        self.n_comp = len(comps)
        self._descs = (ComponentDesc * self.n_comp)(*[component_desc(c) for c in comps])
        mats_p = None
        if inst.materials is not None:
            self._coef = np.ascontiguousarray(inst.materials.coef, dtype=np.float64)
            self._mats = MaterialTables(self._coef.shape[0], self._coef.shape[1],
                                        float(inst.materials.e_min), float(inst.materials.e_max),
                                        self._coef.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
            mats_p = ctypes.byref(self._mats)
        ph_p = None
        if inst.phantom is not None:
            self._vox = np.ascontiguousarray(inst.phantom, dtype=np.uint8)
            nz, ny, nx = self._vox.shape
            self._ph = Phantom(self._vox.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nx, ny, nz)
            if getattr(inst, "mu_scatter", None) is not None:
                self._mus = scatter_table(inst.mu_scatter, self._coef.shape)
                self._ph.mu_scatter = self._mus.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            if getattr(inst, "mu_compton", None) is not None:
                self._muc = scatter_table(inst.mu_compton, self._coef.shape)
                self._ph.mu_compton = self._muc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            ph_p = ctypes.byref(self._ph)
        opt = Options()
        opt.precision = PRECISIONS[precision]
        opt.instr_id = int(inst.instr_id)
        opt.device = int(device)
        opt.block_size = int(block_size)
        opt.blocks_per_sm = int(blocks_per_sm)
        self._alloc = None
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = 0
        if allocator is not None or torch_alloc:
            self._alloc = allocator if allocator is not None else _TorchAllocator(device)
            opt.alloc = self._alloc.alloc_cb
            opt.free = self._alloc.free_cb
        opt.stream = stream
        self.stream = stream
        self.precision = precision
        h = ctypes.c_void_p()
        check(L.mcx_instrument_create(self._descs, self.n_comp, mats_p, ph_p, ctypes.byref(opt),
                                      ctypes.byref(h)))
        self._h = h
        if specialize:
            self.specialize()

    # ---- tracing
    def trace(self, n_rays: int, seed: int):
        check(lib().mcx_trace(self._h, int(n_rays), int(seed)))

    def trace_range(self, ray_begin: int, ray_end: int, seed: int):
        check(lib().mcx_trace_range(self._h, int(ray_begin), int(ray_end), int(seed)))

    def sample_starts(self, ray_begin: int, n: int, seed: int, out):
        """Fill the device tensor `out` (float32, 6*n elements: rows sx, sy,
        E, u, v, w0) with the starts the source draws for rays
        [ray_begin, ray_begin + n)."""
        assert out.is_cuda and out.dtype.is_floating_point and out.numel() >= 6 * n
        check(lib().mcx_sample_starts(self._h, int(ray_begin), int(n), int(seed), out.data_ptr()))

    def trace_starts(self, starts, n: int, ray_base: int = 0, det_w=None):
        """Trace n rays from the device start tensor; `det_w` (device float32
        tensor of n, optional) receives each ray's weight at the last monitor."""
        check(lib().mcx_trace_starts(self._h, starts.data_ptr(), int(n), int(ray_base),
                                     None if det_w is None else det_w.data_ptr()))

    def reset(self):
        check(lib().mcx_monitor_reset(self._h))

    def synchronize(self):
        check(lib().mcx_synchronize(self._h))

    # ---- readout
    def monitor_bins(self, comp: int) -> int:
        n = ctypes.c_size_t()
        check(lib().mcx_monitor_bins(self._h, int(comp), ctypes.byref(n)))
        return int(n.value)

    def specialize(self, enable: bool = True):
        """Trace with a kernel compiled for this instrument's component table
        (constants folded; same arithmetic as the generic kernel)."""
        check(lib().mcx_instrument_specialize(self._h, 1 if enable else 0))

    def kernel_source(self) -> str:
        """The generated source of this instrument's specialised kernel."""
        n = ctypes.c_size_t()
        check(lib().mcx_instrument_source(self._h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        check(lib().mcx_instrument_source(self._h, buf, n.value, None))
        return buf.value.decode()

    def monitor(self, comp: int, out=None):
        """(N uint64, sum_w float64, sum_w2 float64) of monitor `comp`.

        `out` may give the three host arrays to fill (numpy arrays or CPU
        torch tensors, e.g. page-locked ones reused across reads); each needs
        exactly monitor_bins(comp) elements of the matching dtype."""
        nb = self.monitor_bins(comp)
        if out is None:
            out = (np.empty(nb, dtype=np.uint64), np.empty(nb, dtype=np.float64),
                   np.empty(nb, dtype=np.float64))
        ptrs = []
        for a, dt in zip(out, ("uint64", "float64", "float64")):
            ptrs.append(_host_ptr(a, nb, dt))
        check(lib().mcx_monitor_read(self._h, int(comp), *ptrs, nb))
        return tuple(out)

    def monitor_async(self, comp: int, out):
        """Queue the read of monitor `comp` into the three host arrays `out`
        (as for monitor(); page-locked ones let the copies overlap other
        streams' work) on this instrument's stream and return at once; the
        arrays hold the bins after synchronize()."""
        nb = self.monitor_bins(comp)
        ptrs = [_host_ptr(a, nb, dt) for a, dt in zip(out, ("uint64", "float64", "float64"))]
        check(lib().mcx_monitor_read_async(self._h, int(comp), *ptrs, nb))
        return tuple(out)

    def tallies(self) -> dict:
        lost = np.zeros(self.n_comp, dtype=np.float64)
        n_emit = ctypes.c_uint64()
        w0 = ctypes.c_double()
        wend = ctypes.c_double()
        check(lib().mcx_tally_read(self._h, lost.ctypes.data, self.n_comp, ctypes.byref(n_emit),
                                   ctypes.byref(w0), ctypes.byref(wend)))
        return {"lost": lost, "n_emit": int(n_emit.value), "sum_w0": w0.value, "sum_wend": wend.value}

    def monitor_total(self, comp: int) -> tuple:
        """(count, sum w, sum w^2) over every bin of monitor `comp`, reduced on
        the device (mcx_monitor_total)."""
        n = ctypes.c_uint64()
        a = ctypes.c_double()
        b = ctypes.c_double()
        check(lib().mcx_monitor_total(self._h, int(comp), ctypes.byref(n), ctypes.byref(a), ctypes.byref(b)))
        return int(n.value), a.value, b.value

    def loss(self) -> np.ndarray:
        """Weight removed by each component (mcx_loss_read)."""
        lost = np.zeros(self.n_comp, dtype=np.float64)
        check(lib().mcx_loss_read(self._h, lost.ctypes.data, self.n_comp))
        return lost

    def attach(self, proposal, angle: float = 0.0):
        """Draw every later trace's starts from `proposal` (None detaches);
        the proposal must stay alive while attached."""
        L = _proposal_lib()
        check(L.mcx_proposal_attach(self._h, proposal._h if proposal is not None else None,
                                    ctypes.c_float(angle)))
        self._proposal = proposal

    def close(self):
        if getattr(self, "_h", None):
            lib().mcx_instrument_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def batch_trace_static(instruments, budgets, seed: int, chunk_rays: int = 0):
    """Allocation-free batched trace (mcx_batch_trace_static): for callers that
    cannot allocate device memory; at most 512 instruments per call."""
    n = len(instruments)
    if len(budgets) != n:
        raise ValueError(f"{n} instruments but {len(budgets)} budgets")
    hs = (ctypes.c_void_p * n)(*[i._h for i in instruments])
    bud = (ctypes.c_uint64 * n)(*[int(b) for b in budgets])
    check(lib().mcx_batch_trace_static(hs, bud, n, int(chunk_rays), int(seed)))


class Batch:
    """Many instruments traced by one persistent (graph-captured) launch.

    ``instruments`` must share device, precision and stream and outlive the
    batch; ``budgets[i]`` is the ray count of instrument i."""

    def __init__(self, instruments, budgets, chunk_rays: int = 0, block_size: int = 0,
                 blocks_per_sm: int = 0, use_graph: bool = True):
        L = lib()
        self.instruments = list(instruments)
        n = len(self.instruments)
        if len(budgets) != n:
            raise ValueError(f"{n} instruments but {len(budgets)} budgets")
        hs = (ctypes.c_void_p * n)(*[i._h for i in self.instruments])
        self._budgets = (ctypes.c_uint64 * n)(*[int(b) for b in budgets])
        opt = BatchOptions(int(chunk_rays), int(block_size), int(blocks_per_sm), int(bool(use_graph)), 0)
        h = ctypes.c_void_p()
        check(L.mcx_batch_create(hs, self._budgets, n, ctypes.byref(opt), ctypes.byref(h)))
        self._h = h

    def trace(self, seed: int):
        check(lib().mcx_batch_trace(self._h, int(seed)))

    def autotune(self, sample_rays: int, seed: int = 12345) -> dict:
        o = BatchOptions()
        check(lib().mcx_batch_autotune(self._h, int(sample_rays), int(seed), ctypes.byref(o)))
        return {"chunk_rays": o.chunk_rays, "block_size": o.block_size,
                "blocks_per_sm": o.blocks_per_sm, "use_graph": o.use_graph}

    def specialize(self, enable: bool = True):
        """Compile the batch's kernel by instrument families (or go back to
        the generic kernel)."""
        check(lib().mcx_batch_specialize(self._h, int(bool(enable))))

    def items(self) -> int:
        n = ctypes.c_uint64()
        check(lib().mcx_batch_items(self._h, ctypes.byref(n)))
        return int(n.value)

    def synchronize(self):
        self.instruments[0].synchronize()

    def close(self):
        if getattr(self, "_h", None):
            lib().mcx_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ProposalDesc(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("half_u", ctypes.c_float), ("half_v", ctypes.c_float),
                ("x_shift", ctypes.c_float * 4), ("x_scale", ctypes.c_float * 4),
                ("device", ctypes.c_int32), ("reserved", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class TrainOpts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_uint32), ("batch", ctypes.c_uint32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


N_PROPOSAL_PARAMS = 38824


def _proposal_lib():
    L = lib()
    if not getattr(L, "_proposal_ready", False):
        P, vp, u64 = ctypes.POINTER, ctypes.c_void_p, ctypes.c_uint64
        L.mcx_proposal_create.argtypes = [P(ProposalDesc), vp, P(vp)]
        L.mcx_proposal_set_params.argtypes = [vp, vp]
        L.mcx_proposal_get_params.argtypes = [vp, vp]
        L.mcx_proposal_forward.argtypes = [vp, vp, u64, vp]
        L.mcx_proposal_loss_grad.argtypes = [vp, vp, vp, vp, u64, P(ctypes.c_double), vp]
        L.mcx_proposal_train.argtypes = [vp, vp, vp, u64, ctypes.c_float, P(TrainOpts), P(ctypes.c_double)]
        L.mcx_proposal_sample.argtypes = [vp, vp, u64, u64, u64, ctypes.c_float, vp]
        L.mcx_proposal_attach.argtypes = [vp, vp, ctypes.c_float]
        L.mcx_proposal_train_angles.argtypes = [vp, vp, vp, vp, u64, P(TrainOpts), P(ctypes.c_double)]
        L.mcx_proposal_train_angles.restype = ctypes.c_int
        L.mcx_proposal_set_wait_limit.argtypes = [vp, ctypes.c_int64]
        L.mcx_proposal_set_wait_limit.restype = ctypes.c_int
        L.mcx_proposal_destroy.argtypes = [vp]
        L.mcx_proposal_destroy.restype = None
        for name in ("mcx_proposal_create", "mcx_proposal_set_params", "mcx_proposal_get_params",
                     "mcx_proposal_forward", "mcx_proposal_loss_grad", "mcx_proposal_train",
                     "mcx_proposal_sample", "mcx_proposal_attach"):
            getattr(L, name).restype = ctypes.c_int
        L._proposal_ready = True
    return L


class Proposal:
    """Learned importance-sampling proposal for a source's aim point."""

    def __init__(self, alpha: float, half_u: float, half_v: float, x_shift, x_scale,
                 params=None, device: int = 0, stream=None):
        L = _proposal_lib()
        d = ProposalDesc()
        d.alpha, d.half_u, d.half_v = float(alpha), float(half_u), float(half_v)
        d.x_shift[:] = [float(v) for v in x_shift]
        d.x_scale[:] = [float(v) for v in x_scale]
        d.device = int(device)
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = 0
        d.stream = stream
        p = None
        if params is not None:
            self._p0 = np.ascontiguousarray(params, dtype=np.float32)
            assert self._p0.size == N_PROPOSAL_PARAMS
            p = self._p0.ctypes.data
        h = ctypes.c_void_p()
        check(L.mcx_proposal_create(ctypes.byref(d), p, ctypes.byref(h)))
        self._h = h

    def set_params(self, params):
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == N_PROPOSAL_PARAMS
        check(_proposal_lib().mcx_proposal_set_params(self._h, a.ctypes.data))

    def get_params(self) -> np.ndarray:
        a = np.zeros(N_PROPOSAL_PARAMS, dtype=np.float32)
        check(_proposal_lib().mcx_proposal_get_params(self._h, a.ctypes.data))
        return a

    def forward(self, x, out):
        """Network outputs for device rows x (n, 4) into device out (n, 40)."""
        check(_proposal_lib().mcx_proposal_forward(self._h, x.data_ptr(), x.shape[0], out.data_ptr()))

    def loss_grad(self, x, t, w):
        loss = ctypes.c_double()
        g = np.zeros(N_PROPOSAL_PARAMS, dtype=np.float32)
        check(_proposal_lib().mcx_proposal_loss_grad(self._h, x.data_ptr(), t.data_ptr(), w.data_ptr(),
                                                     x.shape[0], ctypes.byref(loss), g.ctypes.data))
        return loss.value, g

    def train(self, starts, det, n: int, angle: float = 0.0, epochs: int = 1, batch: int = 8192,
              lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
              angles=None) -> float:
        """Adam on a history; `angles` (device float tensor of n) gives each
        row its own projection angle instead of `angle`."""
        o = TrainOpts(int(epochs), int(batch), float(lr), float(beta1), float(beta2), float(eps))
        loss = ctypes.c_double()
        L = _proposal_lib()
        if angles is not None:
            check(L.mcx_proposal_train_angles(self._h, starts.data_ptr(), det.data_ptr(), angles.data_ptr(),
                                              int(n), ctypes.byref(o), ctypes.byref(loss)))
        else:
            check(L.mcx_proposal_train(self._h, starts.data_ptr(), det.data_ptr(), int(n),
                                       float(angle), ctypes.byref(o), ctypes.byref(loss)))
        return loss.value

    def set_wait_limit(self, polls: int):
        """Testing: polls before a tensor-core wait gives up (< 0: default)."""
        check(_proposal_lib().mcx_proposal_set_wait_limit(self._h, int(polls)))

    def sample(self, inst: "Instrument", ray_begin: int, n: int, seed: int, out, angle: float = 0.0):
        check(_proposal_lib().mcx_proposal_sample(self._h, inst._h, int(ray_begin), int(n), int(seed),
                                                  float(angle), out.data_ptr()))

    def close(self):
        if getattr(self, "_h", None):
            _proposal_lib().mcx_proposal_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
