"""Pins of the CPU oracle against facts that do not come from the oracle itself:
published known-answer vectors, closed forms, invariants, exact symmetries and
brute force on tiny inputs (no GPU needed)."""

import math
import os

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MM = 1e-3


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v, 16) for v in line.split()])
    return rows


# ------------------------------------------------------------------ RNG
def test_philox_known_answers(orc):
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        assert orc.philox4x32_10(r[0:4], r[4:6]) == r[6:10]


def test_uniform_draw_layout(orc):
    """Draw j of a ray maps onto Philox block words as the draw contract says:
    binary64 draw j = top 53 bits of (w[2(j%2)+1] << 32 | w[2(j%2)]) of block
    j/2; binary32 draw j = top 24 bits of word j%4 of block j/4; counter =
    (id lo, id hi, block, instrument), key = (seed lo, seed hi)."""
    rid, instr, seed = (7 << 32) | 12345, 3, (11 << 32) | 99
    for j in range(8):
        w = orc.philox4x32_10([rid & 0xFFFFFFFF, rid >> 32, j >> 1, instr],
                              [seed & 0xFFFFFFFF, seed >> 32])
        v = (w[2 * (j & 1) + 1] << 32) | w[2 * (j & 1)]
        assert orc.uniform64(rid, instr, seed, j) == (v >> 11) / 2.0**53
        w = orc.philox4x32_10([rid & 0xFFFFFFFF, rid >> 32, j >> 2, instr],
                              [seed & 0xFFFFFFFF, seed >> 32])
        assert orc.uniform32(rid, instr, seed, j) == (w[j & 3] >> 8) / 2.0**24


def test_uniform_statistics(orc):
    """Kolmogorov-Smirnov distance of 20000 draws from U[0,1) in both types."""
    for f in (orc.uniform64, orc.uniform32):
        u = np.sort([f(i, 0, 1, i % 5) for i in range(20000)])
        assert u.min() >= 0.0 and u.max() < 1.0
        d = np.max(np.abs(u - (np.arange(1, u.size + 1) - 0.5) / u.size))
        assert d < 1.63 / math.sqrt(u.size)  # 1% critical value


# ------------------------------------------------------------------ chords
def test_chord_box_closed_forms(orc):
    w = (0.02, 0.03, 0.004)
    # normal incidence through a 4 mm slab
    assert orc.chord_box((0, 0, -1), (0, 0, 1), w) == pytest.approx(0.004, rel=1e-15)
    # oblique: thickness / cos(theta) while inside the lateral extent
    th = 0.3
    k = (math.sin(th), 0.0, math.cos(th))
    assert orc.chord_box((-0.5 * math.tan(th), 0, -0.5), k, w) == pytest.approx(0.004 / math.cos(th), rel=1e-12)
    # starting inside: distance to the exit face
    assert orc.chord_box((0, 0, 0.001), (0, 0, 1), w) == pytest.approx(0.001, rel=1e-12)
    # pointing away or missing laterally
    assert orc.chord_box((0, 0, -1), (0, 0, -1), w) == 0.0
    assert orc.chord_box((0.02, 0, -1), (0, 0, 1), w) == 0.0


def test_chord_cylinder_closed_forms(orc):
    R, h = 0.005, 0.01
    for b in (0.0, 0.001, 0.0049, -0.003):
        # perpendicular to the axis (y) at offset b
        L = orc.chord_cyl((b, 0.0, -0.5), (0, 0, 1), R, h)
        assert L == pytest.approx(2 * math.sqrt(R * R - b * b), rel=1e-12)
    # along the axis, inside: the height
    assert orc.chord_cyl((0.001, -1.0, 0.0), (0, 1, 0), R, h) == pytest.approx(h, rel=1e-12)
    # along the axis, outside the radius: miss
    assert orc.chord_cyl((0.006, -1.0, 0.0), (0, 1, 0), R, h) == 0.0
    # tilted ray through the centre, clipped by the caps: |y| <= h/2 on the
    # line y = z tan(a) gives length h / sin(a) when that is shorter than 2R/cos
    a = 1.2
    k = (0.0, math.sin(a), math.cos(a))
    L = orc.chord_cyl((0.0, -1.0 * math.sin(a), -1.0 * math.cos(a)), k, R, h)
    assert L == pytest.approx(min(h / math.sin(a), 2 * R / math.cos(a)), rel=1e-12)


def test_chord_sphere_and_brute_force(orc):
    R = 0.004
    assert orc.chord_sphere((0.001, 0.002, -1), (0, 0, 1), R) == pytest.approx(
        2 * math.sqrt(R * R - 0.001**2 - 0.002**2), rel=1e-12)
    # random rays: compare every solid with dense sampling along the line
    rng = np.random.default_rng(0)
    t = (np.arange(400000) + 0.5) * (0.04 / 400000)
    for _ in range(20):
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        x = rng.uniform(-0.006, 0.006, 3) - 0.02 * k
        p = x[None, :] + t[:, None] * k[None, :]
        dt = 0.04 / 400000
        box_w = np.array([0.008, 0.006, 0.01])
        inside_box = np.all(np.abs(p) <= box_w / 2, axis=1)
        inside_cyl = (p[:, 0]**2 + p[:, 2]**2 <= 0.005**2) & (np.abs(p[:, 1]) <= 0.004)
        inside_sph = np.sum(p * p, axis=1) <= R * R
        assert orc.chord_box(x, k, box_w) == pytest.approx(inside_box.sum() * dt, abs=3 * dt)
        assert orc.chord_cyl(x, k, 0.005, 0.008) == pytest.approx(inside_cyl.sum() * dt, abs=3 * dt)
        assert orc.chord_sphere(x, k, R) == pytest.approx(inside_sph.sum() * dt, abs=3 * dt)


# ------------------------------------------------------------------ Siddon
def test_siddon_uniform_box_equals_chord(orc):
    vox = np.ones((5, 4, 3), dtype=np.uint8)
    v = 0.001
    mu = np.array([0.0, 250.0])
    rng = np.random.default_rng(1)
    for _ in range(50):
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        x = rng.uniform(-0.001, 0.001, 3) - 0.01 * k
        tau = orc.siddon_tau(x, k, vox, v, mu)
        L = orc.chord_box(x, k, (3 * v, 4 * v, 5 * v))
        assert tau == pytest.approx(250.0 * L, rel=1e-12, abs=1e-12)


def test_siddon_axis_aligned_rows(orc):
    """A ray along x through voxel row (j, k) integrates that row exactly."""
    rng = np.random.default_rng(2)
    vox = rng.integers(0, 4, size=(4, 3, 6)).astype(np.uint8)
    mu = np.array([0.0, 10.0, 100.0, 1000.0])
    v = 0.5e-3
    for k in range(4):
        for j in range(3):
            y = -1.5 * v + (j + 0.5) * v
            z = -2.0 * v + (k + 0.5) * v
            tau = orc.siddon_tau((-1.0, y, z), (1.0, 0.0, 0.0), vox, v, mu)
            assert tau == pytest.approx(v * mu[vox[k, j, :]].sum(), rel=1e-12)


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_siddon_brute_force(orc, n):
    rng = np.random.default_rng(10 + n)
    vox = rng.integers(0, 8, size=(n, n, n)).astype(np.uint8)
    mu = rng.uniform(0, 300, size=8)
    v = 1e-3
    half = 0.5 * n * v
    M = 200000
    for _ in range(8):
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        x = rng.uniform(-half, half, 3) - 3 * half * k
        span = 6 * half
        t = (np.arange(M) + 0.5) * (span / M)
        p = x[None, :] + t[:, None] * k[None, :]
        idx = np.floor((p + half) / v).astype(int)
        ok = np.all((idx >= 0) & (idx < n), axis=1)
        i = idx[ok]
        ref = mu[vox[i[:, 2], i[:, 1], i[:, 0]]].sum() * (span / M)
        tau = orc.siddon_tau(x, k, vox, v, mu)
        assert tau == pytest.approx(ref, abs=mu.max() * 6 * 3 * span / M)


def test_siddon_corner_and_face_rays(orc):
    vox = np.arange(8, dtype=np.uint8).reshape(2, 2, 2)
    mu = np.arange(8, dtype=np.float64) * 10.0
    v = 1.0
    # along the main diagonal through the shared corner: half in voxel 0, half in 7
    k = np.ones(3) / math.sqrt(3)
    tau = orc.siddon_tau(-2 * k, k, vox, v, mu)
    assert tau == pytest.approx(math.sqrt(3) * (mu[0] + mu[7]), rel=1e-12)
    # outside the grid entirely
    assert orc.siddon_tau((5, 5, -5), (0, 0, 1), vox, v, mu) == 0.0


# ------------------------------------------------------------------ fixed-step march (Sec. 3.3)
def _march_direct(x, k, vox, v, s, mu):
    """The fixed-step rule written out in binary64 floating point: steps of
    v/s from the grid entry, each weighted by the voxel of its end point, the
    last one cut at the exit.  Returns (tau, smallest distance of an end point
    from a voxel face, in voxels)."""
    nz, ny, nx = vox.shape
    n = np.array([nx, ny, nz])
    half = 0.5 * n * v
    lo, hi = 0.0, np.inf
    for i in range(3):
        if k[i] != 0.0:
            t1, t2 = (-half[i] - x[i]) / k[i], (half[i] - x[i]) / k[i]
            lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
        elif abs(x[i]) > half[i]:
            return 0.0, np.inf
    if hi <= lo:
        return 0.0, np.inf
    h = v / s
    N = math.ceil((hi - lo) / h)
    tau, margin = 0.0, np.inf
    for j in range(1, N + 1):
        q = (x + (lo + j * h) * k + half) / v
        f = np.floor(q)
        margin = min(margin, float(np.min(np.minimum(q - f, f + 1 - q))))
        idx = np.clip(f.astype(int), 0, n - 1)
        ln = h if j < N else (hi - lo) - (N - 1) * h
        tau += mu[vox[idx[2], idx[1], idx[0]]] * ln
    return tau, margin


@pytest.mark.parametrize("s", [1.0, 3.0, 7.5])
def test_march_uniform_box_sums_the_chord(orc, s):
    """In one material the step lengths add up to the chord, whatever the step."""
    vox = np.ones((5, 4, 3), dtype=np.uint8)
    v = 0.001
    mu = np.array([0.0, 250.0])
    rng = np.random.default_rng(21)
    for _ in range(50):
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        x = rng.uniform(-0.001, 0.001, 3) - 0.01 * k
        L = orc.chord_box(x, k, (3 * v, 4 * v, 5 * v))
        assert orc.march_tau(x, k, vox, v, s, mu) == pytest.approx(250.0 * L, rel=1e-12, abs=1e-12)
    assert orc.march_tau((5, 5, -5), (0, 0, 1), vox, v, s, mu) == 0.0


@pytest.mark.parametrize("s", [1, 3, 4])
def test_march_matches_the_rule_written_out(orc, s):
    """The 32.32 fixed-point march samples the same voxels as the rule in
    plain floating point, wherever no end point lies within 1e-6 voxel of a face."""
    rng = np.random.default_rng(30 + s)
    vox = rng.integers(0, 8, size=(6, 5, 7)).astype(np.uint8)
    mu = rng.uniform(0, 300, size=8)
    v = 1e-3
    checked = 0
    for _ in range(60):
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        x = rng.uniform(-2e-3, 2e-3, 3) - 0.02 * k
        ref, margin = _march_direct(x, k, vox, v, s, mu)
        if margin < 1e-6:
            continue
        checked += 1
        assert orc.march_tau(x, k, vox, v, s, mu) == pytest.approx(ref, rel=1e-12, abs=1e-15)
    assert checked >= 50


def test_march_converges_to_the_line_integral(orc):
    """Each step differs from the exact integral only where it crosses a voxel
    face: |march - Siddon| <= (faces crossed + 2) * step * max |mu_a - mu_b|,
    so the gap closes as the steps shrink."""
    rng = np.random.default_rng(40)
    vox = rng.integers(0, 8, size=(8, 8, 8)).astype(np.uint8)
    mu = rng.uniform(0, 300, size=8)
    v = 1e-3
    dmu = mu.max() - mu.min()
    gaps = {s: [] for s in (1, 3, 10, 30, 100)}
    for _ in range(40):
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        x = rng.uniform(-3e-3, 3e-3, 3) - 0.02 * k
        exact = orc.siddon_tau(x, k, vox, v, mu)
        L = orc.chord_box(x, k, (8 * v, 8 * v, 8 * v))
        faces = L * np.abs(k).sum() / v + 3
        for s in gaps:
            gap = abs(orc.march_tau(x, k, vox, v, s, mu) - exact)
            assert gap <= (faces + 2) * (v / s) * dmu
            gaps[s].append(gap)
    mean = {s: float(np.mean(g)) for s, g in gaps.items()}
    assert mean[100] < mean[10] < mean[1]


def test_march_trace_weights_follow_the_march(orc):
    """A trace through a marched phantom (steps of 1/3 voxel): each detected
    weight is w0 exp(-tau) with tau the fixed-step rule written out above,
    on the ray's own line (binary32 direction, widened), wherever that rule
    is unambiguous (end points >= 1e-4 voxel from a face)."""
    rng = np.random.default_rng(5)
    vox = rng.integers(0, 2, size=(5, 6, 4)).astype(np.uint8)
    spec = wl.edxct_instrument(nx=4, ny=6, nz=5, voxel=10 * MM, n_det=1, det_px=16, pix=6.4 * MM,
                               ne=8, phantom=vox)
    spec.components[1]["march"] = 3
    n = 3000
    st = orc.sample_starts(spec, 0, n, 11)
    _, det_w = orc.trace_starts(spec, st)
    ph = spec.components[1]
    f32 = np.float32
    dz = f32(spec.components[0]["target_dist"])
    checked = 0
    for i in range(n):
        if det_w[i] <= 0.0:
            continue
        sx, sy, E, tx, ty, w0 = (f32(st[r][i]) for r in range(6))
        dx, dy = f32(tx - sx), f32(ty - sy)
        ln = f32(np.sqrt(f32(f32(f32(dx * dx) + f32(dy * dy)) + f32(dz * dz))))
        il = f32(f32(1.0) / ln)
        k = np.array([f32(dx * il), f32(dy * il), f32(dz * il)], dtype=np.float64)
        x = np.array([float(sx), float(sy), 0.0]) - np.array(ph["pos"])
        mus = np.array([orc.mu(spec, m, float(E), 32) for m in range(2)])
        tau, margin = _march_direct(x, k, vox, ph["voxel"], 3, mus)
        if margin < 1e-4:
            continue
        assert det_w[i] == pytest.approx(float(w0) * math.exp(-tau), rel=1e-12)
        checked += 1
    assert checked > n // 4


# ------------------------------------------------------------------ tables
def test_mu_table_nodes_and_edge(orc):
    inst = wl.absorption_instrument()
    a, b = 1.6e6, 2.0
    for E in (20.0, 35.5, 59.9, 60.0, 61.3, 119.9):
        jump = 5.0 if E >= 60.0 else 1.0
        exact = a * jump / E**3 + b
        # node energies on a 0.1 keV grid: the table is exact there
        got = orc.mu(inst, 0, E)
        assert got == pytest.approx(exact, rel=1e-9 if abs(E - round(E, 1)) < 1e-12 else 1e-3)
    # the K-edge sits on a cell boundary: x5 jump of the photoelectric term
    below = orc.mu(inst, 0, 60.0 - 1e-9)
    above = orc.mu(inst, 0, 60.0)
    assert above - b == pytest.approx(5 * (below - b), rel=1e-6)
    # between nodes the table interpolates linearly (convexity: above the curve)
    assert orc.mu(inst, 0, 20.05) >= a / 20.05**3 + b


# ------------------------------------------------------------------ full traces
def test_slit_acceptance_closed_form(orc):
    """Fraction of flat-slit rays through the 0.5 mm slit: 1 - 8R/(3pi) + R^2/(2pi)."""
    inst = wl.flat_slit_instrument()
    n = 200000
    p = 1.0 - 8 * 0.5 / (3 * math.pi) + 0.25 / (2 * math.pi)
    for mode in (64, 32):
        r = orc.trace(inst, 0, n, 1, mode, threads=4)
        N, sw, sw2 = r.monitor(2)
        z = (N.sum() - n * p) / math.sqrt(n * p * (1 - p))
        assert abs(z) < 5
        assert r.lost[1] == n - N.sum()            # every loss is at the slit
        assert (sw == N).all() and (sw2 == N).all()  # flat source: w = 1


def test_wide_slit_passes_everything(orc):
    """A slit of side >= 1 mm at the midplane accepts every ray (|xs+xt| <= 1 mm)."""
    inst = wl.flat_slit_instrument(slit_w=1.0 * MM)
    r = orc.trace(inst, 0, 20000, 5, 64)
    assert r.monitor(2)[0].sum() == 20000
    assert r.lost.sum() == 0.0


def test_flat_slit_images(orc):
    """PSD hits lie on the 1x1 mm target (central 50x50 pixels); the energy
    monitor is flat (chi-square over 200 bins)."""
    inst = wl.flat_slit_instrument()
    r = orc.trace(inst, 0, 100000, 1, 64, threads=4)
    N = r.monitor(2)[0].reshape(100, 100)
    assert N[25:75, 25:75].sum() == N.sum()
    Ne = r.monitor(3)[0]
    assert Ne.sum() == N.sum()
    exp_ = Ne.sum() / 200
    chi2 = ((Ne - exp_) ** 2 / exp_).sum()
    assert chi2 < 199 + 5 * math.sqrt(2 * 199)


def test_rotation_frames_exact(orc):
    """Turning the PSD by +90 deg about z (exact matrix) permutes its image:
    local x = lab y, local y = -lab x."""
    inst = wl.flat_slit_instrument()
    rot = (0.0, -1.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 1.0)
    inst2 = wl.flat_slit_instrument()
    inst2.components[2] = dict(inst2.components[2], rot=rot)
    a = orc.trace(inst, 0, 50000, 4, 64).monitor(2)[0].reshape(100, 100)
    b = orc.trace(inst2, 0, 50000, 4, 64).monitor(2)[0].reshape(100, 100)
    # b[iy_l, ix_l] with ix_l = iy_lab and iy_l = 99 - ix_lab
    assert (b == a.T[::-1, :]).all()
    assert not (b == a).all()


def test_rotated_whole_instrument(orc):
    """Placing every component relative to a source turned by +90 deg about z
    leaves every local coordinate, hence every image, unchanged."""
    inst = wl.flat_slit_instrument()
    rot = (0.0, -1.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 1.0)
    inst2 = wl.flat_slit_instrument()
    inst2.components[0] = dict(inst2.components[0], rot=rot, pos=(0.01, -0.02, 0.3))
    for i in range(1, 4):
        inst2.components[i] = dict(inst2.components[i], relative_to=0)
    a = orc.trace(inst, 0, 30000, 9, 64)
    b = orc.trace(inst2, 0, 30000, 9, 64)
    for c in (2, 3):
        assert (a.monitor(c)[0] == b.monitor(c)[0]).all()


def test_partition_and_threads_invariance(orc):
    inst = wl.absorption_instrument(nx=16, ne=16)
    full = orc.trace(inst, 0, 30000, 2, 64)
    parts = orc.trace(inst, 0, 11111, 2, 64)
    parts.add(orc.trace(inst, 11111, 30000, 2, 64))
    thr = orc.trace(inst, 0, 30000, 2, 64, threads=3)
    for other in (parts, thr):
        assert (other.N == full.N).all()
        np.testing.assert_allclose(other.sw, full.sw, rtol=1e-12)
        assert other.n_emit == full.n_emit


def test_instrument_id_and_seed_change_stream(orc):
    inst = wl.absorption_instrument(nx=8, ne=8)
    a = orc.trace(inst, 0, 5000, 2, 64).N
    inst.instr_id = 1
    b = orc.trace(inst, 0, 5000, 2, 64).N
    c = orc.trace(wl.absorption_instrument(nx=8, ne=8), 0, 5000, 3, 64).N
    assert not (a == b).all() and not (a == c).all()


def _weight_conservation(r, rel=1e-12):
    assert r.sum_w0 == pytest.approx(r.lost.sum() + r.sum_wend, rel=rel)


@pytest.mark.parametrize("mode", [64, 32])
def test_weight_conservation(orc, mode):
    for inst in (wl.flat_slit_instrument(), wl.absorption_instrument(nx=32, ne=32),
                 wl.ct_instrument(n=32, voxel=4 * MM, n_pix=32, pix=8 * MM, ne=16, window=1.5)):
        _weight_conservation(orc.trace(inst, 0, 4000, 3, mode))


def test_kramers_weights_have_unit_mean(orc):
    """w0 = f(E)/mean(f) with E uniform: E[w0] = 1 (z-test)."""
    inst = wl.absorption_instrument(nx=8, ne=8)
    n = 100000
    r = orc.trace(inst, 0, n, 7, 64, threads=4)
    # per-ray w0 variance: E[f^2]/fbar^2 - 1, from the closed-form moments
    lo, hi, e0 = 20.0, 120.0, 120.0
    fbar = (e0 * math.log(hi / lo) - (hi - lo)) / (hi - lo)
    f2 = (e0 * e0 * (1 / lo - 1 / hi) - 2 * e0 * math.log(hi / lo) + (hi - lo)) / (hi - lo)
    sd = math.sqrt(f2 / fbar**2 - 1.0)
    assert abs(r.sum_w0 / n - 1.0) < 5 * sd / math.sqrt(n)


def test_monoenergetic_pencil_beer_lambert(orc):
    """A zero-width target makes every ray travel along +z; with a zero-width
    energy band every ray has E = 40 keV: each detected weight is exactly
    exp(-mu d) through a d = 3 mm slab."""
    mats = wl.tabulate_materials([(1.6e6, 2.0, 60.0, 5.0)], 20.0, 120.0, 1000)
    comps = [
        wl.component("source", shape="point", spectrum="flat", e_min=40.0, e_max=40.0,
                     target_dist=1.0, target_w=0.0, target_h=0.0),
        wl.component("abs_box", pos=(0, 0, 0.5), wx=0.01, wy=0.01, wz=0.003, material=0),
        wl.component("mon_psd", pos=(0, 0, 1.0), nx=2, ny=2, xmin=-1e-3, xmax=1e-3,
                     ymin=-1e-3, ymax=1e-3),
    ]
    inst = wl.Instrument(components=comps, materials=mats)
    r = orc.trace(inst, 0, 1000, 1, 64)
    N, sw, sw2 = r.monitor(2)
    mu = 1.6e6 / 40.0**3 + 2.0
    assert N.sum() == 1000
    assert sw.sum() == pytest.approx(1000 * math.exp(-mu * 0.003), rel=1e-13)
    assert sw2.sum() == pytest.approx(1000 * math.exp(-2 * mu * 0.003), rel=1e-13)


def _cylinder_expected_weight(inst, nq=800, nL=3000):
    """Mean detected weight per ray of the absorption instrument by quadrature:
    E_{u,v,E}[ f(E)/fbar * exp(-mu(E) L(u,v)) ], with L the chord of the line
    from the point source through the aim point (u, v, D) in the cylinder,
    written with the line parameter lambda (point = lambda (u, v, D))."""
    src, cyl = inst.components[0], inst.components[1]
    D, W = src["target_dist"], src["target_w"]
    R, H = cyl["radius"], cyl["height"]
    lo, hi, e0 = src["e_min"], src["e_max"], src["e0"]
    fbar = (e0 * math.log(hi / lo) - (hi - lo)) / (hi - lo)
    coef = inst.materials.coef[0]
    ncell = coef.shape[0]
    de = (hi - lo) / ncell
    gx, gw = np.polynomial.legendre.leggauss(6)
    E = (lo + (np.arange(ncell)[:, None] + 0.5 * (gx[None, :] + 1)) * de).ravel()
    wE = np.tile(gw * 0.5 * de, ncell) / (hi - lo)
    muE = coef[np.repeat(np.arange(ncell), gx.size), 0] + coef[np.repeat(np.arange(ncell), gx.size), 1] * E
    fE = (e0 - E) / E / fbar
    Ls = np.linspace(0.0, 2.2 * R, nL)
    g = np.array([(wE * fE * np.exp(-muE * L)).sum() for L in Ls])
    # quadrant of the aim rectangle (the chord is even in u and v)
    uu = (np.arange(nq) + 0.5) * (0.5 * W / nq)
    u, v = np.meshgrid(uu, uu, indexing="ij")
    A = u * u + D * D
    disc = D**4 - A * (D * D - R * R)
    ok = disc > 0
    sq = np.sqrt(np.where(ok, disc, 0.0))
    l1, l2 = (D * D - sq) / A, (D * D + sq) / A
    lcap = np.where(v > 0, 0.5 * H / np.maximum(v, 1e-300), np.inf)
    l2 = np.minimum(l2, lcap)
    length = np.where(ok & (l2 > l1), (l2 - l1) * np.sqrt(u * u + v * v + D * D), 0.0)
    return float(np.interp(length, Ls, g).mean())


def test_absorption_transmission_quadrature(orc):
    inst = wl.absorption_instrument(nx=16, ne=16)
    n = 200000
    r = orc.trace(inst, 0, n, 2, 64, threads=4)
    N, sw, sw2 = r.monitor(2)
    assert N.sum() == n  # the detector covers the whole shadow
    m = sw.sum() / n
    sd = math.sqrt((sw2.sum() / n - m * m) / n)
    expect = _cylinder_expected_weight(inst)
    assert abs(m - expect) < 5 * sd, (m, expect, sd)


def test_mode32_statistics(orc):
    """The binary32 path samples its own (24-bit) rays: totals agree statistically."""
    inst = wl.absorption_instrument(nx=64, ne=64)
    a = orc.trace(inst, 0, 50000, 2, 64)
    b = orc.trace(inst, 0, 50000, 2, 32)
    assert a.N.sum() == b.N.sum() == 50000
    # 32-bit sampling moves every ray slightly, so compare totals and spectra
    assert np.abs(a.sw.sum() - b.sw.sum()) / a.sw.sum() < 2e-2


def _two_monitor_instrument(order, restore):
    src = wl.component("source", shape="point", spectrum="flat", e_min=10.0, e_max=30.0,
                       target_dist=1.0, target_w=2 * MM, target_h=2 * MM)
    mons = {z: wl.component("mon_psd", pos=(0, 0, z), nx=8, ny=8, xmin=-1 * MM, xmax=1 * MM,
                            ymin=-1 * MM, ymax=1 * MM, restore=restore) for z in (0.6, 0.8)}
    return wl.Instrument(components=[src] + [mons[z] for z in order], name="two_monitors")


@pytest.mark.parametrize("mode", [64, 32])
def test_restoring_monitors_see_every_ray_in_any_order(orc, mode):
    """A restoring monitor (McXtrace's restore_xray) leaves the ray as it
    found it: two such monitors give the same images in either order, and the
    ray is never lost.  Without restore, the nearer monitor listed second
    lies behind the ray and absorbs it."""
    n = 20_000
    a = orc.trace(_two_monitor_instrument((0.6, 0.8), True), 0, n, 3, mode)
    b = orc.trace(_two_monitor_instrument((0.8, 0.6), True), 0, n, 3, mode)
    assert np.array_equal(a.monitor(1)[0], b.monitor(2)[0])     # z = 0.6
    assert np.array_equal(a.monitor(2)[0], b.monitor(1)[0])     # z = 0.8
    assert a.monitor(1)[0].sum() > 0.2 * n and b.lost.sum() == 0.0
    c = orc.trace(_two_monitor_instrument((0.8, 0.6), False), 0, n, 3, mode)
    assert c.monitor(2)[0].sum() == 0 and c.lost[2] == pytest.approx(n, rel=1e-12)


def _bin32(v, lo, hi, n):
    """The monitor bin rule in binary32, vectorised: inv = n / (hi - lo)
    formed in binary64 and rounded once, then (v - lo) * inv in binary32
    (numpy's binary32 operations round each result once); -1 outside."""
    f32 = np.float32
    inv = f32(float(n) / (hi - lo))
    f = (np.asarray(v, dtype=f32) - f32(lo)) * inv
    ok = (f >= f32(0)) & (f < f32(n))
    return np.where(ok, np.floor(f), -1).astype(np.int64)


def test_edxct_arc_counts_match_direct_projection(orc):
    """The paper's EDXCT arc of five tilted, restoring line detectors (no
    phantom attenuation: vacuum voxels).  Each sampled ray is projected onto
    each detector plane independently of the oracle, twice:
    * in binary32 along the operation sequence of the arithmetic contract
      (direction, binary64 frames, binary32 plane propagation, the bin rule):
      every ray lands in the same pixel and energy bin as the oracle's, with
      no tolerance, edge rays included;
    * in binary64 (the geometry without the contract's roundings): it agrees
      with the binary32 projection except for rays whose binary64 hit lies
      within 64 binary32 ulps of 2.5 m (the arc's radius) of a pixel or
      aperture edge."""
    spec = wl.edxct_instrument(nx=4, ny=6, nz=5, voxel=10 * MM, det_px=16, pix=6.4 * MM, ne=8,
                               phantom=np.zeros((5, 6, 4), dtype=np.uint8))
    n = 30_000
    st32 = orc.sample_starts(spec, 0, n, 7)
    res, _ = orc.trace_starts(spec, st32)
    st = st32.astype(np.float64)
    src = spec.components[0]
    f32 = np.float32
    # binary32 direction: d = aim - source, k = d (1 / sqrt((dx dx + dy dy) + dz dz))
    dx, dy, dz = st32[3] - st32[0], st32[4] - st32[1], np.full(n, f32(src["target_dist"]))
    il = f32(1) / np.sqrt((dx * dx + dy * dy) + dz * dz)
    k32 = np.stack([dx * il, dy * il, dz * il], axis=1).astype(np.float64)
    Rs = np.array(src["rot"] if src["rot"] is not None else np.eye(3).ravel()).reshape(3, 3)
    os_ = np.array(src["pos"])
    sl = np.stack([st[0], st[1], np.zeros(n)], axis=1)
    X = np.stack([os_[i] + ((Rs[i, 0] * sl[:, 0] + Rs[i, 1] * sl[:, 1]) + Rs[i, 2] * sl[:, 2])
                  for i in range(3)], axis=1)
    K = np.stack([(Rs[i, 0] * k32[:, 0] + Rs[i, 1] * k32[:, 1]) + Rs[i, 2] * k32[:, 2] for i in range(3)], axis=1)
    # binary64 geometry of the same rays
    d = np.stack([st[3] - st[0], st[4] - st[1], np.full(n, src["target_dist"])], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p0 = np.stack([st[0], st[1], np.zeros(n)], axis=1)
    slack = 64 * 2.0**-24 * 2.5
    total = disagree = 0
    for c in range(2, 2 + 5):
        m = spec.components[c]
        R = np.array(m["rot"]).reshape(3, 3)
        o = np.array(m["pos"])
        e = X - o
        xl = np.stack([(R[0, i] * e[:, 0] + R[1, i] * e[:, 1]) + R[2, i] * e[:, 2] for i in range(3)], axis=1)
        kl = np.stack([(R[0, i] * K[:, 0] + R[1, i] * K[:, 1]) + R[2, i] * K[:, 2] for i in range(3)], axis=1)
        x32, q32 = xl.astype(f32), kl.astype(f32)
        with np.errstate(divide="ignore", invalid="ignore"):
            t = -x32[:, 2] / q32[:, 2]
        reach = (q32[:, 2] != 0) & (t >= 0)
        hx = x32[:, 0] + t * q32[:, 0]
        hy = x32[:, 1] + t * q32[:, 1]
        ix = _bin32(hx, m["xmin"], m["xmax"], m["nx"])
        iy = _bin32(hy, m["ymin"], m["ymax"], m["ny"])
        ie = _bin32(st32[2], m["e_min"], m["e_max"], m["ne"])
        ok = reach & (ix >= 0) & (iy >= 0) & (ie >= 0)
        ref = np.zeros(m["nx"] * m["ny"] * m["ne"], dtype=np.int64)
        np.add.at(ref, (iy[ok] * m["nx"] + ix[ok]) * m["ne"] + ie[ok], 1)
        assert np.array_equal(res.monitor(c)[0].astype(np.int64), ref), c
        total += int(ref.sum())
        # binary64 geometry: differs only next to an edge
        R64 = R
        xl64 = (p0 - o) @ R64
        kl64 = d @ R64
        t64 = -xl64[:, 2] / kl64[:, 2]
        x64 = xl64[:, 0] + t64 * kl64[:, 0]
        y64 = xl64[:, 1] + t64 * kl64[:, 1]
        jx = np.floor((x64 - m["xmin"]) * m["nx"] / (m["xmax"] - m["xmin"]))
        jy = np.floor((y64 - m["ymin"]) * m["ny"] / (m["ymax"] - m["ymin"]))
        ok64 = (t64 > 0) & (jx >= 0) & (jx < m["nx"]) & (jy >= 0) & (jy < m["ny"]) & (ie >= 0)
        differ = (ok64 != ok) | (ok & ok64 & ((jx != ix) | (jy != iy)))
        ex = np.linspace(m["xmin"], m["xmax"], m["nx"] + 1)
        ey = np.linspace(m["ymin"], m["ymax"], m["ny"] + 1)
        dist = np.minimum(np.abs(x64[:, None] - ex[None, :]).min(axis=1),
                          np.abs(y64[:, None] - ey[None, :]).min(axis=1))
        assert np.all(dist[differ] <= slack), (c, dist[differ].max())
        disagree += int(differ.sum())
    assert total > 0.9 * n                  # the fan lands on the arc
    assert disagree <= 0.01 * total


# ------------------------------------------------------------------ aim direction
# The unit direction of a sampled ray (source point to aim point, A2 of the
# method's steps) is formed by one square root, one reciprocal and three
# products.  Pin: every component equals the exact d/|d| of the (mode-rounded)
# inputs to a few units in the last place, so that |k| = 1 and the ray lands
# on its aim point; a dropped term, a wrong sign, a swapped component or a
# binary32 step in the binary64 mode each fail it.
_AIM_ULPS = 6


def _aim_cases():
    rng = np.random.default_rng(41)
    cases = [(0.0, 0.0, 0.0, 0.0, 1.0), (1e-4, -2e-4, 1e-4, -2e-4, 0.5),   # straight along z
             (0.0, 0.0, 0.3, 0.0, 1.0), (0.0, 0.0, 0.0, -0.3, 1.0)]
    for _ in range(400):   # disk sources onto a 1 mm target at 1 m
        cases.append(tuple(rng.uniform(-5e-4, 5e-4, 4)) + (1.0,))
    for _ in range(400):   # cone beams onto a 256 mm detector at 1 m
        cases.append(tuple(rng.uniform(-5e-6, 5e-6, 2)) + tuple(rng.uniform(-0.2, 0.2, 2)) + (1.0,))
    for _ in range(200):   # steep rays: aim far off axis at a short distance
        cases.append(tuple(rng.uniform(-1e-3, 1e-3, 2)) + tuple(rng.uniform(-2.0, 2.0, 2)) +
                     (float(rng.uniform(0.01, 0.1)),))
    return cases


def _aim_violations(orc, mode, lib_=None):
    """Cases whose direction breaks the bound (returned as a list)."""
    import decimal
    from decimal import Decimal
    decimal.getcontext().prec = 60
    u = Decimal(2) ** (-53 if mode == 64 else -24)
    bad = []
    for c in _aim_cases():
        if mode == 32:
            c = tuple(float(np.float32(v)) for v in c)
        sx, sy, tx, ty, tz = (Decimal(v) for v in c)
        d = (tx - sx, ty - sy, tz)
        n = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]).sqrt()
        exact = [di / n for di in d]
        kf = orc.aim_direction(mode, *c, lib_=lib_)
        if not all(np.isfinite(kf)):
            bad.append(("not finite", c))
            continue
        k = [Decimal(v) for v in kf]
        if any(abs(ki - ei) > _AIM_ULPS * u * abs(ei) for ki, ei in zip(k, exact)):
            bad.append(("component", c))
            continue
        # the ray's point at z = tz against the aim point
        for i, (s, t) in enumerate(((sx, tx), (sy, ty))):
            land = s + tz * k[i] / k[2]
            if abs(land - t) > 4 * _AIM_ULPS * u * (abs(s) + abs(t) + tz * abs(k[i] / k[2])):
                bad.append(("landing", c))
    return bad


@pytest.mark.parametrize("mode", [64, 32])
def test_aim_direction_is_unit_and_hits_the_aim_point(orc, mode):
    assert _aim_violations(orc, mode) == []
    k = orc.aim_direction(mode, 0.0, 0.0, 0.0, 0.0, 1.0)
    assert k == [0.0, 0.0, 1.0]


_AIM_LEN = "const REAL len = SQRTR(dx * dx + dy * dy + dz * dz);"
_AIM_D = "const REAL dx = tx - sx, dy = ty - sy, dz = tz;"
_AIM_K1 = "k[1] = dy * il;"
_AIM_IL = "const REAL il = (REAL)1 / len;"
AIM_PLANTS = {
    "dropped_z_term": [("orc_core.inc", _AIM_LEN, "const REAL len = SQRTR(dx * dx + dy * dy);")],
    "wrong_sign": [("orc_core.inc", _AIM_D, "const REAL dx = sx - tx, dy = ty - sy, dz = tz;")],
    "swapped_component": [("orc_core.inc", _AIM_K1, "k[1] = dx * il;")],
    "binary32_reciprocal": [("orc_core.inc", _AIM_IL, "const REAL il = (REAL)(1.0f / (float)len);")],
}


@pytest.mark.parametrize("plant", sorted(AIM_PLANTS))
def test_each_planted_aim_mistake_fails_the_pin(orc, plant, tmp_path):
    L = orc.build_variant(AIM_PLANTS[plant], str(tmp_path / plant))
    modes = (64,) if plant == "binary32_reciprocal" else (64, 32)
    for mode in modes:
        assert _aim_violations(orc, mode, lib_=L), f"the planted mistake {plant!r} passes in mode {mode}"
