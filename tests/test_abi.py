"""The C ABI library loads, exports every entry point its headers declare, and
rejects invalid instruments on the host before touching a GPU (no GPU needed)."""

import ctypes
import glob
import math
import os
import re

import pytest

from paper_2410_08747_gb300 import mcx
from paper_2410_08747_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2410_08747_gb300 import build
    build.build()
    return mcx.lib()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(mcx_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert "mcx_instrument_create" in names and "mcx_trace" in names
    for n in names:
        assert hasattr(L, n), n


def _create(L, comps, mats=None, ph=None, **optkw):
    descs = (mcx.ComponentDesc * len(comps))(*[mcx.component_desc(c) for c in comps])
    opt = mcx.Options()
    for k, v in optkw.items():
        setattr(opt, k, v)
    h = ctypes.c_void_p()
    st = L.mcx_instrument_create(descs, len(comps), mats, ph, ctypes.byref(opt), ctypes.byref(h))
    return st, h


def test_rejects_invalid_descriptions(L):
    good = wl.flat_slit_instrument().components
    cases = []
    cases.append([good[1], good[0]] + good[2:])                      # source not first
    bad = [dict(c) for c in good]
    bad[2]["relative_to"] = 3                                          # forward reference
    cases.append(bad)
    bad = [dict(c) for c in good]
    bad[1] = dict(bad[1], xmin=math.nan)                               # NaN parameter
    cases.append(bad)
    bad = [dict(c) for c in good]
    bad[2] = dict(bad[2], nx=0)                                        # empty monitor
    cases.append(bad)
    bad = [dict(c) for c in good]
    bad[1] = dict(bad[1], rot=(2, 0, 0, 0, 1, 0, 0, 0, 1))            # not a rotation
    cases.append(bad)
    bad = [dict(c) for c in good]
    bad[0] = dict(bad[0], spectrum="kramers", e0=5.0)                  # e0 < e_max
    cases.append(bad)
    for comps in cases:
        st, h = _create(L, comps)
        assert st == -1, comps
        assert len(L.mcx_last_error()) > 0
    # absorber without material tables
    st, _ = _create(L, wl.absorption_instrument().components)
    assert st == -1
    # unknown precision, bad block size
    st, _ = _create(L, good, precision=7)
    assert st == -1
    st, _ = _create(L, good, block_size=100)
    assert st == -1


def test_null_arguments(L):
    assert L.mcx_trace_range(None, 0, 10, 1) == -1
    assert L.mcx_monitor_reset(None) == -1
    assert L.mcx_monitor_read(None, 0, None, None, None, 0) == -1
    assert L.mcx_monitor_read_async(None, 0, None, None, None, 0) == -1
    L.mcx_instrument_destroy(None)


def test_batch_proposal_and_start_calls_reject_bad_arguments(L):
    """Host-side validation of the batch, ray-start and proposal entry points
    (every case returns MCX_ERR_INVALID before selecting a device)."""
    out = ctypes.c_void_p()
    assert L.mcx_batch_create(None, None, 0, None, ctypes.byref(out)) == -1
    assert L.mcx_batch_create(None, None, 1, None, None) == -1
    assert L.mcx_batch_trace(None, 1) == -1
    assert L.mcx_sample_starts(None, 0, 10, 1, None) == -1
    assert L.mcx_trace_starts(None, None, 10, 0, None) == -1

    def prop(**kw):
        d = mcx.ProposalDesc()
        d.alpha, d.half_u, d.half_v = 0.1, 1e-3, 1e-3
        d.x_scale[:] = [1.0] * 4
        for k, v in kw.items():
            setattr(d, k, v)
        h = ctypes.c_void_p()
        return L.mcx_proposal_create(ctypes.byref(d), None, ctypes.byref(h))
    assert prop(alpha=0.0) == -1
    assert prop(alpha=1.5) == -1
    assert prop(half_u=0.0) == -1
    assert prop(half_v=-1.0) == -1
    d = mcx.ProposalDesc()
    d.alpha, d.half_u, d.half_v = 0.1, 1e-3, 1e-3
    d.x_scale[:] = [1.0, math.nan, 1.0, 1.0]
    assert L.mcx_proposal_create(ctypes.byref(d), None, ctypes.byref(out)) == -1
    o = mcx.TrainOpts(1, 64, 1e-3, 0.9, 0.999, 1e-8)
    assert L.mcx_proposal_train(None, None, None, 0, ctypes.c_float(0.0), ctypes.byref(o), None) == -1
    assert b"NULL" in L.mcx_last_error()


def _mats_ph(spec):
    coef = __import__("numpy").ascontiguousarray(spec.materials.coef, dtype="float64")
    mats = mcx.MaterialTables(coef.shape[0], coef.shape[1], spec.materials.e_min, spec.materials.e_max,
                              coef.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    ph = None
    keep = [coef]
    if spec.phantom is not None:
        import numpy as np
        vox = np.ascontiguousarray(spec.phantom, dtype=np.uint8)
        nz, ny, nx = vox.shape
        ph = mcx.Phantom(vox.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nx, ny, nz)
        keep.append(vox)
        if spec.mu_scatter is not None:
            mus = mcx.scatter_table(spec.mu_scatter, coef.shape)
            ph.mu_scatter = mus.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            keep.append(mus)
    return mats, ph, keep


def test_rejects_invalid_lens_source_march_and_scatter(L):
    """The parameters of the focusing instrument, the fixed-step march and
    the scattering phantom are checked on the host before any GPU call."""
    import numpy as np
    foc = wl.focusing_instrument()
    mats, _, keep = _mats_ph(foc)
    bad_lens = [dict(n_lenses=0), dict(n_lenses=5000), dict(aperture=-1e-3), dict(delta0=0.5),
                dict(material=3), dict(radius=0.0)]
    for kw in bad_lens:
        comps = [dict(c) for c in foc.components]
        comps[1] = dict(comps[1], **kw)
        st, _ = _create(L, comps, ctypes.byref(mats))
        assert st == -1, kw
    comps = [dict(c) for c in foc.components]
    comps[0] = dict(comps[0], div_x=-1e-6)                  # negative divergence
    assert _create(L, comps, ctypes.byref(mats))[0] == -1
    comps = [dict(c) for c in foc.components]
    comps[0] = dict(comps[0], sigma_e=-1.0)                 # negative energy spread
    assert _create(L, comps, ctypes.byref(mats))[0] == -1
    blk = wl.scatter_block()
    mats2, ph2, keep2 = _mats_ph(blk)
    comps = [dict(c) for c in blk.components]
    comps[1] = dict(comps[1], march=65)                     # above 64 steps per voxel
    assert _create(L, comps, ctypes.byref(mats2), ctypes.byref(ph2))[0] == -1
    comps = [dict(c) for c in blk.components]
    comps[1] = dict(comps[1], march=0)                      # scattering without the march
    assert _create(L, comps, ctypes.byref(mats2), ctypes.byref(ph2))[0] == -1
    ph2.mu_scatter = ctypes.POINTER(ctypes.c_double)()      # scattering without coefficients
    assert _create(L, blk.components, ctypes.byref(mats2), ctypes.byref(ph2))[0] == -1
    nc = blk.materials.n_cell
    neg = mcx.scatter_table(np.array([0.0, -1.0, 2.0]), (3, nc))
    ph2.mu_scatter = neg.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert _create(L, blk.components, ctypes.byref(mats2), ctypes.byref(ph2))[0] == -1
    assert "scattering" in L.mcx_last_error().decode()
    # a line that is >= 0 at a cell's lower end but crosses zero inside it
    cross = mcx.scatter_table(np.array([0.0, 1.0, 2.0]), (3, nc))
    cross[2, 7] = (21.5, -1.0)     # cell 7 is [21.4, 21.6) keV: 0.1 at its lower end, -0.1 at its upper
    ph2.mu_scatter = cross.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert _create(L, blk.components, ctypes.byref(mats2), ctypes.byref(ph2))[0] == -1
    assert "on every cell" in L.mcx_last_error().decode()
    nan = mcx.scatter_table(np.array([0.0, 1.0, 2.0]), (3, nc))
    nan[1, 3, 1] = np.nan
    ph2.mu_compton = nan.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ph2.mu_scatter = keep2[-1].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert _create(L, blk.components, ctypes.byref(mats2), ctypes.byref(ph2))[0] == -1
    assert "Compton" in L.mcx_last_error().decode()
    # more than 32 materials: the two per-thread columns would not fit
    coef33 = np.ascontiguousarray(np.repeat(blk.materials.coef[1:2], 33, 0))
    mats33 = mcx.MaterialTables(33, nc, blk.materials.e_min, blk.materials.e_max,
                                coef33.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    mus33 = mcx.scatter_table(np.ones(33), (33, nc))
    ph2.mu_scatter = mus33.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ph2.mu_compton = ctypes.POINTER(ctypes.c_double)()
    assert _create(L, blk.components, ctypes.byref(mats33), ctypes.byref(ph2))[0] == -1
    assert "32 materials" in L.mcx_last_error().decode()
