"""Benchmark: traced rays/s and Monte Carlo figure of merit on one GB300.

Workload: the absorption instrument (point source, Kramers spectrum 20-120
keV, cone onto a 10 mm cylinder of the synthetic K-edge material, 128x128
pixel x 256 energy-bin detector at 1 m), 1e8 rays per step.  The chosen form
(binary32 propagation, binary64 frames and sums), traced by the kernel the
library compiles for this instrument, is the timed value; the plain binary64
form runs beside it for the figure-of-merit comparison
FOM = 1 / (relative variance x seconds) of the detector-integrated weight,
and the generic (uncompiled) kernel is timed on the same steps.

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
(N > 1 under torch.distributed.run: every rank traces its own ray-id range,
no collective on the data path).  Prints one JSON line on rank 0.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "traced rays/s and MC FOM 1/(rel.var*s), chosen vs plain form, same GB300"
WORKLOAD = "absorption instrument: point source, Kramers 20-120 keV, 10 mm K-edge cylinder, 128x128x256 detector"
N_RAYS = 100_000_000
SEED0 = 2


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax),
                       reasons=sorted(reasons), samples=len(sm))
        return out


def relvar_of_sum(n, sw, sw2):
    """Relative variance of the mean weight per ray from its first two moments."""
    m = sw / n
    var = max(sw2 / n - m * m, 0.0) / n
    return var / (m * m) if m > 0 else float("inf")


def cpu_oracle_rate(spec, n, threads, mode=64, seed=SEED0):
    from oracle import oracle
    comp = oracle.Compiled(spec)
    oracle.trace(spec, 0, 1000, seed, mode, threads=1, compiled=comp)  # warm
    t0 = time.perf_counter()
    oracle.trace(spec, 0, n, seed, mode, threads=threads, compiled=comp)
    return n / (time.perf_counter() - t0)


def reference_arm(args):
    """The CPU oracle timed on the host cores: each step a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2410_08747_gb300 import workloads as wl
    spec = wl.absorption_instrument()
    cores = os.cpu_count() or 1
    sample = 2_000_000
    for _ in range(args.warmup):
        cpu_oracle_rate(spec, sample // 10, cores)
    rates = [cpu_oracle_rate(spec, sample, cores) for _ in range(args.steps)]
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sample / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rays_per_step": sample},
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample} rays of the workload per step, binary64 oracle, "
                                       f"{cores} host threads"},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rays", type=int, default=N_RAYS)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workload shapes (measured after the timed region)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch

    from paper_2410_08747_gb300 import mcx, shard
    from paper_2410_08747_gb300 import workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = local
    stream = torch.cuda.current_stream(dev)
    n = args.rays
    spec = wl.absorption_instrument()

    # both forms trace with the kernel compiled for this instrument (its
    # component table folded into the code); the compilation happens once,
    # before any timing, as a user would compile an instrument before a run
    t0 = time.perf_counter()
    chosen = mcx.Instrument(spec, precision="mixed", device=dev, specialize=True)
    compile_s = time.perf_counter() - t0
    plain = mcx.Instrument(spec, precision="fp64", device=dev, specialize=True)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=f"cuda:{dev}")

    def ray_range(step):
        # every rank and step traces its own ray ids
        return shard.step_range(rank, world, step, n)

    def timed_steps(inst, steps, warmup, label_seed):
        ms = []
        for s in range(warmup):
            b, e = ray_range(10_000 + s)
            inst.trace_range(b, e, label_seed)
        torch.cuda.synchronize(dev)
        for s in range(steps):
            flush.zero_()                                    # evict L2 between steps
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b, e = ray_range(s)
            ev0.record(stream)
            inst.trace_range(b, e, label_seed)
            ev1.record(stream)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        return ms

    # ---- chosen form: timed region with barrier + synchronize on both sides
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(dev) as clk:
        ms_chosen = timed_steps(chosen, args.steps, args.warmup, SEED0)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    total_ms = sum(ms_chosen)
    if dist:
        t = torch.tensor([total_ms], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * n * args.steps / (total_ms / 1e3)

    # ---- plain form and FOM (same rays per step)
    chosen.reset()
    plain_steps = max(2, min(args.steps, 4))
    ms_plain = timed_steps(plain, plain_steps, 1, SEED0)
    chosen.reset()
    plain.reset()
    chosen.trace_range(0, n, SEED0 + 100)
    plain.trace_range(0, n, SEED0 + 100)
    fom = {}
    for name, inst, ms in (("chosen", chosen, ms_chosen), ("plain", plain, ms_plain)):
        N, sw, sw2 = inst.monitor(2)
        rv = relvar_of_sum(n, float(sw.sum()), float(sw2.sum()))
        sec = statistics.median(ms) / 1e3
        fom[name] = {"rays_per_s": n / sec, "relvar": rv, "seconds": sec, "fom": 1.0 / (rv * sec)}
    fom["ratio"] = fom["chosen"]["fom"] / fom["plain"]["fom"]

    # ---- the generic kernel (table in shared memory) on the same steps
    generic = mcx.Instrument(spec, precision="mixed", device=dev)
    ms_generic = timed_steps(generic, plain_steps, 1, SEED0)
    generic.close()
    fom["tally"] = "detector-integrated sum of weights, relvar from (N, sum w, sum w^2)"

    # ---- end to end through the C ABI with host buffers: per step create
    # (H2D of the description and tables), trace, read the full detector back
    # (D2H) into page-locked arrays and read the tallies.  Serial: one step
    # after the other.  Overlapped (the `e2e` value): consecutive steps
    # alternate two streams and two host buffers, and each step's detector
    # read (mcx_monitor_read_async: device split, then DMA) runs while the
    # next step traces, as a caller reading every step's detector would run
    # it; the timed region spans every step's create, trace, read and tallies
    e2e_steps = max(2, min(args.steps, 4))
    nb = chosen.monitor_bins(2)
    h2d = (len(spec.components) * 224 + spec.materials.coef.nbytes)
    d2h = nb * 24 + 8 * (len(spec.components) + 2)

    def pinned():
        return tuple(torch.empty(nb * 8, dtype=torch.uint8, pin_memory=True).numpy().view(dt)
                     for dt in (np.uint64, np.float64, np.float64))

    host = pinned()
    e2e_t = []
    for s in range(e2e_steps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        g = mcx.Instrument(spec, precision="mixed", device=dev, specialize=True)
        b, e = ray_range(20_000 + s)
        g.trace_range(b, e, SEED0)
        g.monitor(2, out=host)
        g.tallies()
        t1 = time.perf_counter()
        g.close()
        if s > 0:
            e2e_t.append(t1 - t0)
    e2e_serial = world * n / statistics.median(e2e_t)
    streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    hosts = [host, pinned()]

    def e2e_overlapped(k, first):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        prev = None
        for s in range(k):
            g = mcx.Instrument(spec, precision="mixed", device=dev, specialize=True,
                               stream=streams[s % 2].cuda_stream)
            b, e = ray_range(first + s)
            g.trace_range(b, e, SEED0)
            g.monitor_async(2, hosts[s % 2])
            if prev is not None:
                prev.synchronize()
                prev.tallies()
                prev.close()
            prev = g
        prev.synchronize()
        prev.tallies()
        prev.close()
        return time.perf_counter() - t0

    # as many overlapped steps as the device-timed region has, so that the
    # pipeline's fill (the first create) and drain (the last read) weigh as
    # they would over a run of that length
    e2e_overlapped(2, 30_000)   # warm-up
    e2e_k = max(2, args.steps)
    e2e_rate = world * n * e2e_k / e2e_overlapped(e2e_k, 30_100)

    # ---- roofline of the dominant kernel (the fused tracer)
    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "rays_per_step": n, "precision": "mixed",
                       "kernel": "compiled for the instrument (run-time, constants folded)",
                       "l2": "flushed between timed steps (512 MiB write)",
                       "parallelism": f"replicas x{world}"},
            "plain_fp64_rays_per_s": fom["plain"]["rays_per_s"],
            "generic_kernel_rays_per_s": n / (statistics.median(ms_generic) / 1e3),
            "compile_seconds": compile_s,
            "fom": fom,
            "e2e": {"value": e2e_rate, "unit": "rays/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_k, "serial_steps": e2e_steps,
                    "mode": "consecutive steps on two streams, each step's detector read overlapping the next trace"},
            "e2e_serial_rays_per_s": e2e_serial,
            "gpu_launches": args.steps,
            "clocks": clocks}
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    with ClockSampler(dev) as clk_peaks:
        peaks = measure_peaks(mcx, dev, DETECTOR_BYTES_ABSORPTION)
    peaks["clocks"] = clk_peaks.summary()
    line["measured_peaks"] = peaks
    line["roofline"] = roofline(n, total_ms / args.steps, peaks, n_sm)
    if not args.no_extras and world == 1:
        chosen.close()
        plain.close()
        flush = None
        torch.cuda.empty_cache()
        line["configs"] = extra_configs(mcx, wl, torch, dev, stream, peaks)
    if rank == 0 and not args.no_cpu:
        cores = os.cpu_count() or 1
        sample = 20_000_000
        rate = cpu_oracle_rate(spec, sample, cores)
        one = cpu_oracle_rate(spec, sample // 10, 1)
        line["cpu_baseline"] = {"value": rate, "unit": "rays/s", "cores": cores, "kind": "oracle",
                                "sample": f"{sample} rays (ids 0..{sample}) of the workload, "
                                          f"binary64 oracle, {cores} host threads",
                                "single_thread": {"value": one, "unit": "rays/s",
                                                  "sample": f"{sample // 10} rays, one host thread "
                                                            "(the paper's baseline convention)"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# Algorithmic work per ray of the mixed form on the absorption instrument,
# counted from the draw-and-arithmetic contract, per hardware unit:
# * lane operations (each arithmetic, logic, compare, conversion, division,
#   square root, exponential and atomic operation once): Philox block 100,
#   uniforms 9, aim point and energy 7, direction 11, Kramers weight 3, frame
#   changes 20, cylinder chord 30, mu(E) and attenuation 10, detector plane,
#   bins and scoring 31, tallies 12;
# * Philox4x32-10 blocks: one (three binary32 draws: aim u, v and energy);
# * binary64 operations on the FP64 pipe: the frame changes into the cylinder
#   and the detector frames (one subtraction each: both sit on the beam
#   axis with identity rotations), the widening of the hit's weight and its
#   square;
# * monitor hits: one per ray that reaches the detector (every ray: the
#   detector covers the whole cone), three global atomic adds each.
OPS_PER_RAY_ABSORPTION = 233
PHILOX_PER_RAY_ABSORPTION = 1
FP64_PER_RAY_ABSORPTION = 4
HITS_PER_RAY_ABSORPTION = 1.0
DETECTOR_BYTES_ABSORPTION = 128 * 128 * 256 * 24

# DRAM bytes (read + write) of one timed 1e8-ray launch of the compiled
# absorption kernel, from one ncu capture of this benchmark's first timed
# launch (dram__bytes_read.sum + dram__bytes_write.sum); None whenever the
# kernel has changed since the capture.
TRAFFIC_BYTES_PER_LAUNCH = 63.60e6


def measure_peaks(mcx, dev, footprint):
    """The library's microbenchmarks (mcx_peak_measure) on this GPU, now:
    FFMA, IMAD and DFMA lane operations/s, Philox blocks/s, and monitor hits/s
    (three atomics each) at the detector's footprint, random bins."""
    out = {}
    for k in ("ffma", "imad", "philox", "dfma"):
        out[k] = mcx.peak_measure(k, dev)
    out["hit"] = mcx.peak_measure("hit", dev, footprint)
    out["hit_footprint_bytes"] = footprint
    return out


def roofline(n, ms, peaks, n_sm):
    """Roofline of the fused tracer kernel over its hardware units (the
    kernel is not a dense contraction): per unit, the algorithmic work of a
    launch / its CUDA-event time against that unit's measured peak; the
    binding unit is the one with the largest fraction."""
    sec = ms / 1e3
    legs = {
        "issue": (OPS_PER_RAY_ABSORPTION * n / sec, peaks["ffma"], "lane ops/s (FFMA-measured issue rate)"),
        "philox": (PHILOX_PER_RAY_ABSORPTION * n / sec, peaks["philox"], "Philox blocks/s"),
        "fp64": (FP64_PER_RAY_ABSORPTION * n / sec, peaks["dfma"], "FP64 ops/s (DFMA-measured)"),
        "atomics": (HITS_PER_RAY_ABSORPTION * n / sec, peaks["hit"],
                    "monitor hits/s, 3 atomics each (measured at the detector's footprint)"),
    }
    fr = {k: a / p for k, (a, p, _) in legs.items()}
    bound = max(fr, key=fr.get)
    a, p, _ = legs[bound]
    scale, unit = {"issue": (1e12, "Tops/s"), "philox": (1e9, "G Philox blocks/s"),
                   "fp64": (1e12, "T FP64 ops/s"), "atomics": (1e9, "G monitor hits/s")}[bound]
    hbm = measured_peaks().get("hbm_gbs")
    out = {"bound": "atomic" if bound == "atomics" else "alu", "unit_bound": bound,
           "achieved": a / scale, "peak": p / scale, "unit": unit,
           "frac": fr[bound], "traffic": TRAFFIC_BYTES_PER_LAUNCH,
           "peak_source": "measured now on this GPU by the library's microbenchmarks (mcx_peak_measure)",
           "legs": {k: {"achieved": legs[k][0], "peak": legs[k][1], "frac": fr[k], "unit": legs[k][2]}
                    for k in legs},
           "per_ray": {"lane_ops": OPS_PER_RAY_ABSORPTION, "philox_blocks": PHILOX_PER_RAY_ABSORPTION,
                       "fp64_ops": FP64_PER_RAY_ABSORPTION, "hits": HITS_PER_RAY_ABSORPTION},
           "n_sm": n_sm,
           "algorithmic_bytes": DETECTOR_BYTES_ABSORPTION}
    if TRAFFIC_BYTES_PER_LAUNCH and hbm:
        out["hbm_frac_of_traffic"] = TRAFFIC_BYTES_PER_LAUNCH / sec / 1e9 / float(hbm)
    return out


def _events(torch, stream):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def learned_ct(mcx, wl, torch, dev, timed):
    """The learned proposal on the CT projection (window 1.5x the detector),
    trained over projection angles and judged against the plain binary64
    form and the mixed form with the uniform sampler.

    * Histories: 36 projection angles k pi/36 (the phantom rotated about
      y), 2.78e6 plain-traced rays each (1e8 in all), the rows interleaved
      across angles; one network for all angles (the angle is a network
      input, given per row), one epoch of Adam on 65536-row batches.
    * Evaluation at an angle outside the training set (0.3 rad): for each
      form K = 32 runs under seeds 100..131, each timed with CUDA events;
      the primary tally (the detector-integrated sum of weights, reduced on
      the device) of each run gives the relative variance of one run by batch
      means, cross-checked against the moment formula; the secondary tally is
      the median per-bin relative variance of one run over the bins above
      1e-3 of the largest.
    * FOM = 1 / (relvar x seconds per run), training excluded and amortised
      over the 32 runs, and the break-even ray count of the learned form
      against the uniform mixed form with training counted."""
    import numpy as np
    from paper_2410_08747_gb300 import stats
    phantom = wl.make_phantom(256, seed=3)

    def spec_at(th):
        return wl.ct_instrument(angle=th, window=1.5, spot=10e-6, phantom=phantom)

    spec = spec_at(0.0)
    src = spec.components[0]
    e_mid, e_half = 0.5 * (src["e_min"] + src["e_max"]), 0.5 * (src["e_max"] - src["e_min"])
    angles = [k * math.pi / 36 for k in range(36)]
    n_per, batch = 100_000_000 // len(angles), 65536
    n_hist = n_per * len(angles)
    prop = mcx.Proposal(0.1, 0.5 * src["target_w"], 0.5 * src["target_h"], [0, 0, e_mid, 0],
                        [1 / 10e-6, 1 / 10e-6, 1 / e_half, 1 / math.pi],
                        params=wl.proposal_init(0).astype("float32"), device=dev)
    st = torch.empty((6, n_hist), dtype=torch.float32, device=f"cuda:{dev}")
    det = torch.empty(n_hist, dtype=torch.float32, device=f"cuda:{dev}")
    ang = torch.empty(n_hist, dtype=torch.float32, device=f"cuda:{dev}")
    t_hist = 0.0
    for k, th in enumerate(angles):
        base = mcx.Instrument(spec_at(th), precision="mixed", device=dev)
        s_ = torch.empty(6 * n_per, dtype=torch.float32, device=f"cuda:{dev}")
        d_ = det[k * n_per:(k + 1) * n_per]
        t_hist += timed(lambda: (base.sample_starts(0, n_per, 6 + k, s_), base.trace_starts(s_, n_per, 0, d_)))
        st[:, k * n_per:(k + 1) * n_per].copy_(s_.view(6, n_per))
        ang[k * n_per:(k + 1) * n_per].fill_(th)
        base.close()
        del s_
    # interleave the angles (row j of angle k to position j * 36 + k): every
    # 65536-row batch holds ~1820 rows of each angle (rows of one angle are
    # independent draws, so this mixes as well as a random shuffle)
    t0 = time.perf_counter()
    na = len(angles)
    st = st.view(6, na, n_per).transpose(1, 2).contiguous().view(6, n_hist)
    det = det.view(na, n_per).t().contiguous().view(n_hist)
    ang = ang.view(na, n_per).t().contiguous().view(n_hist)
    torch.cuda.synchronize(dev)
    t_mix = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss = prop.train(st.view(-1), det, n_hist, epochs=1, batch=batch, lr=3e-3, angles=ang)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    del st, det, ang
    th_eval = 0.3
    spec_eval = spec_at(th_eval)
    # the sampler alone (prop_tc_kernel: two 128 x 128 layers and the 128 x 48
    # head on the tensor cores, 2 x 38.6 k = 77 kFLOP per start counting the
    # 4 -> 128 layer too), timed on 2^23-start chunks against the measured
    # BF16 burst peak
    g = mcx.Instrument(spec_eval, precision="mixed", device=dev)
    n_s = 1 << 23
    buf = torch.empty(6 * n_s, dtype=torch.float32, device=f"cuda:{dev}")
    prop.sample(g, 0, n_s, 98, buf, th_eval)
    t_s = statistics.median([timed(lambda: prop.sample(g, r * n_s, n_s, 98, buf, th_eval)) for r in range(1, 6)])
    flop = SAMPLER_FLOP_PER_START * n_s / t_s
    peak = measured_peaks().get("bf16_tflops")
    sampler = {"starts": n_s, "starts_per_s": n_s / t_s, "tflops": flop / 1e12,
               "flop_per_start": SAMPLER_FLOP_PER_START,
               "frac_of_measured_bf16_burst": (flop / 1e12 / float(peak)) if peak else None}
    g.close()
    del buf
    K, seeds = 32, list(range(100, 132))
    forms = {"plain_fp64": ("fp64", 20_000_000, False), "mixed_uniform": ("mixed", 100_000_000, False),
             "mixed_learned": ("mixed", 100_000_000, True)}
    res = {}
    for name, (prec, n, learned) in forms.items():
        g = mcx.Instrument(spec_eval, precision=prec, device=dev, specialize=True)
        if learned:
            g.attach(prop, th_eval)
        g.trace_range(0, n // 10, 99)               # warm-up (compilation, first launch)
        secs, tots, rv_mom = [], [], []
        for k, seed in enumerate(seeds):
            g.reset()
            secs.append(timed(lambda: g.trace_range(0, n, seed)))
            c, sw, sw2 = g.monitor_total(2)
            tots.append(sw / n)
            rv_mom.append(stats.relvar_of_sum(n, sw, sw2))
            if k == 0:
                N_, swb, sw2b = g.monitor(2)
                secondary = stats.secondary_relvar(n, swb, sw2b)
        mean, rv = stats.relvar_batch_means(tots)
        sec = statistics.median(secs)
        res[name] = {"rays": n, "runs": K, "seeds": [seeds[0], seeds[-1]], "seconds": sec,
                     "rays_per_s": n / sec, "mean_w": mean, "relvar": rv,
                     "relvar_moments": float(np.mean(rv_mom)), "relvar_secondary": secondary,
                     "fom": stats.fom(rv, sec)}
        g.close()
    pl, mu, le = res["plain_fp64"], res["mixed_uniform"], res["mixed_learned"]
    setup = t_hist + t_mix + t_train
    le["fom_training_amortised_over_runs"] = stats.fom_amortised(le["relvar"], le["seconds"], setup, K)
    le["fom_training_in_one_run"] = stats.fom(le["relvar"], le["seconds"] + setup)
    # one network serves every projection of a scan (the angle is an input):
    # a 360-projection scan shares the training
    le["fom_training_amortised_over_360_projections"] = stats.fom_amortised(le["relvar"], le["seconds"], setup, 360)
    res["z_learned_vs_plain"] = stats.z_score(le["mean_w"], le["relvar"] / K, pl["mean_w"], pl["relvar"] / K)
    res["z_uniform_vs_plain"] = stats.z_score(mu["mean_w"], mu["relvar"] / K, pl["mean_w"], pl["relvar"] / K)
    res["ratio_learned_vs_plain"] = le["fom"] / pl["fom"]
    res["ratio_learned_vs_mixed_uniform"] = le["fom"] / mu["fom"]
    res["ratio_learned_amortised_vs_plain"] = le["fom_training_amortised_over_runs"] / pl["fom"]
    res["ratio_learned_amortised_vs_mixed_uniform"] = le["fom_training_amortised_over_runs"] / mu["fom"]
    res["ratio_learned_scan_amortised_vs_mixed_uniform"] = (
        le["fom_training_amortised_over_360_projections"] / mu["fom"])
    res["secondary_relvar_learned_over_uniform"] = le["relvar_secondary"] / mu["relvar_secondary"]
    res["break_even_rays_vs_mixed_uniform"] = stats.break_even_rays(
        le["relvar"], le["rays"], le["rays_per_s"], setup, mu["relvar"], mu["rays"], mu["rays_per_s"])
    res["batched_scan"] = learned_batch_scan(mcx, wl, dev, timed, spec_at, prop, stats, setup)
    res["sampler"] = sampler
    res["training"] = {"angles": len(angles), "histories": n_hist, "history_seconds": t_hist,
                       "interleave_seconds": t_mix, "train_seconds": t_train, "epochs": 1, "batch": batch,
                       "last_loss": loss,
                       "note": "the FOM set-up time is history + interleave + train seconds",
                       "eval_angle": th_eval,
                       "learned_path": "proposal attached to the instrument: sampled and traced in "
                                       "2^23-ray chunks"}
    prop.close()
    return res


# Algorithmic operations of the CT walk: per voxel crossed, one byte load
# (or word extraction), a three-way minimum, the next crossing's add, the
# depth's multiply-add and the offset step (6); per ray the source,
# direction, frames, detector and tallies of the absorption count (233 less
# its chord 30 and attenuation 10 = 193) plus the walk's set-up (entry voxel,
# per-axis increments and first crossings, ~30) and the per-ray mu(E) of the
# eight materials (~10): 233.
CT_OPS_PER_VOXEL = 6
CT_OPS_PER_RAY = 233
# Multiply-adds of the learned proposal per start, times two: 4 x 128 +
# 128 x 128 + 128 x 128 + 128 x 40 weights plus the biases (38,824
# parameters, 2 FLOP each).
SAMPLER_FLOP_PER_START = 2 * 38_824


def learned_batch_scan(mcx, wl, dev, timed, spec_at, prop, stats, setup, n_proj=8, rays=25_000_000, runs=8):
    """The chosen form of the scope's target, learned + batched + FP32: a
    scan of n_proj projections at angles outside the training set
    (0.3 + k pi / n_proj), rays per projection, traced as one batch
    (mcx_batch_trace, the proposal attached to every projection), against
    the same scan with the uniform sampler as one graph-launched batch.
    runs repeats under seeds 200.. give each projection's relative variance
    by batch means; FOM = 1 / (mean relvar x seconds per scan), the learned
    one also with the network's one-off set-up (`setup` seconds) charged to
    this scan and amortised over a 360-projection scan (45 such scans)."""
    import numpy as np
    th = [0.3 + k * math.pi / n_proj for k in range(n_proj)]
    out = {}
    for name, learned in (("mixed_uniform", False), ("mixed_learned", True)):
        insts = [mcx.Instrument(spec_at(t), precision="mixed", device=dev) for t in th]
        if learned:
            for g, t in zip(insts, th):
                g.attach(prop, t)
        b = mcx.Batch(insts, [rays] * n_proj, chunk_rays=1 << 18)
        b.specialize()
        b.trace(199)                                   # warm-up (and graph capture)
        secs, tots = [], [[] for _ in th]
        for k in range(runs):
            for g in insts:
                g.reset()
            secs.append(timed(lambda: b.trace(200 + k)))
            for j, g in enumerate(insts):
                tots[j].append(g.monitor_total(2)[1] / rays)
        rv = float(np.mean([stats.relvar_batch_means(t)[1] for t in tots]))
        sec = statistics.median(secs)
        out[name] = {"projections": n_proj, "rays_per_projection": rays, "runs": runs,
                     "seconds_per_scan": sec, "rays_per_s": n_proj * rays / sec,
                     "mean_relvar_per_projection": rv, "fom": stats.fom(rv, sec)}
        b.close()
        for g in insts:
            g.close()
    le, un = out["mixed_learned"], out["mixed_uniform"]
    le["fom_setup_charged_to_scan"] = stats.fom(le["mean_relvar_per_projection"], le["seconds_per_scan"] + setup)
    le["fom_setup_amortised_360_projections"] = stats.fom_amortised(
        le["mean_relvar_per_projection"], le["seconds_per_scan"], setup, 360 // n_proj)
    out["fom_ratio_learned_vs_uniform"] = le["fom"] / un["fom"]
    out["fom_ratio_learned_setup_charged_vs_uniform"] = le["fom_setup_charged_to_scan"] / un["fom"]
    out["fom_ratio_learned_setup_amortised_360_vs_uniform"] = le["fom_setup_amortised_360_projections"] / un["fom"]
    out["path"] = "one mcx_batch_trace per scan; phantom instruments staged in 2^23-ray waves, aim-tile ordered"
    return out


def extra_configs(mcx, wl, torch, dev, stream, peaks):
    """The other workload shapes, each measured once (CUDA events): the flat
    slit instrument, the CT projection (plain and mixed), the batched CT-scan
    workload (one graph-replayed persistent launch after autotuning) and the
    learned proposal's figure of merit against the plain form."""
    out = {}

    def timed(fn):
        e0, e1 = _events(torch, stream)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    # flat slit instrument, 1e6 rays per run
    spec = wl.flat_slit_instrument()
    r = {}
    for prec in ("mixed", "fp64"):
        for kern in ("generic", "compiled"):
            g = mcx.Instrument(spec, precision=prec, device=dev, specialize=kern == "compiled")
            g.trace(1_000_000, 1)
            sec = timed(lambda: g.trace_range(0, 1_000_000, 2))
            r[f"{prec}_{kern}"] = {"rays_per_s": 1e6 / sec, "rays": 1_000_000}
            g.close()
    out["flat_slit_1e6"] = r

    # CT projection, 256^3 phantom, 256x256x128 detector; the voxels a ray
    # crosses in the grid (the walk's work unit) counted in closed form on a
    # sample of the device-drawn starts: 1 + sum_i |floor(exit_i) - floor(entry_i)|
    spec = wl.ct_instrument()
    r = {}
    import numpy as np
    ph = spec.components[1]
    g = mcx.Instrument(spec, precision="mixed", device=dev)
    ns = 200_000
    stt = torch.empty(6 * ns, dtype=torch.float32, device=dev)
    g.sample_starts(0, ns, 4, stt)
    st = stt.view(6, ns).cpu().numpy().astype(np.float64)
    g.close()
    d = np.stack([st[3] - st[0], st[4] - st[1], np.full(ns, spec.components[0]["target_dist"])], 1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p0 = np.stack([st[0], st[1], np.zeros(ns)], 1) - np.array(ph["pos"])
    h = 0.5 * ph["nx"] * ph["voxel"]
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (-h - p0) / d
        t2 = (h - p0) / d
    lo = np.nanmax(np.minimum(t1, t2), axis=1)
    hi = np.nanmin(np.maximum(t1, t2), axis=1)
    hit = hi > lo
    ent = (p0[hit] + lo[hit, None] * d[hit] + h) / ph["voxel"]
    ext = (p0[hit] + hi[hit, None] * d[hit] + h) / ph["voxel"]
    n_ax = ph["nx"] - 1
    cross = 1 + np.abs(np.clip(np.floor(ext), 0, n_ax) - np.clip(np.floor(ent), 0, n_ax)).sum(axis=1)
    voxels_per_ray = float(cross.sum() / ns)
    for prec, n in (("mixed", 200_000_000), ("fp64", 20_000_000)):
        for kern in ("generic", "compiled"):
            g = mcx.Instrument(spec, precision=prec, device=dev, specialize=kern == "compiled")
            g.trace_range(0, n // 10, 4)
            sec = timed(lambda: g.trace_range(10**10, 10**10 + n, 4))
            r[f"{prec}_{kern}"] = {"rays_per_s": n / sec, "rays": n,
                                   "voxel_steps_per_s": n / sec * voxels_per_ray}
            g.close()
    r["voxels_per_ray"] = voxels_per_ray
    mc = r["mixed_compiled"]
    issue = (CT_OPS_PER_VOXEL * mc["voxel_steps_per_s"] + CT_OPS_PER_RAY * mc["rays_per_s"])
    r["roofline_mixed_compiled"] = {
        "ops_per_voxel_step": CT_OPS_PER_VOXEL, "ops_per_ray": CT_OPS_PER_RAY,
        "issue_frac_of_measured_ffma": issue / peaks["ffma"],
        "hits_frac_of_measured_at_201MB": mc["rays_per_s"] / mcx.peak_measure("hit", dev, 256 * 256 * 128 * 24)}
    out["ct_256"] = r

    # the paper's EDXCT line scanner: 350 x 250 x 100 mm water in 1 mm voxels,
    # five tilted 1 x 128-pixel, 128-bin line detectors on an arc at 2.5 m
    # (exact walk), and the paper's own traversal: steps of 1/3 voxel, each
    # weighted by the voxel at its end (detector sum relative to the walk's
    # on the same rays)
    spec = wl.edxct_instrument()
    marched = wl.edxct_instrument()
    marched.components[1]["march"] = 3
    r = {}
    det_sum = {}
    mons = [c for c, comp in enumerate(spec.components) if comp["type"].startswith("mon_")]
    for prec, n, kern, s in (("mixed", 100_000_000, "compiled", 0), ("mixed", 100_000_000, "generic", 0),
                             ("fp64", 10_000_000, "compiled", 0), ("mixed", 100_000_000, "compiled", 3),
                             ("mixed", 100_000_000, "generic", 3), ("fp64", 10_000_000, "compiled", 3)):
        g = mcx.Instrument(marched if s else spec, precision=prec, device=dev, specialize=kern == "compiled")
        g.trace_range(0, n // 10, 4)
        sec = timed(lambda: g.trace_range(10**10, 10**10 + n, 4))
        key = f"{prec}_{kern}" + (f"_march{s}" if s else "")
        r[key] = {"rays_per_s": n / sec, "rays": n}
        if kern == "compiled":
            det_sum[(prec, s)] = float(sum(g.monitor(c)[1].sum() for c in mons))
            if s:
                r[key]["detector_sum_vs_walk"] = det_sum[(prec, s)] / det_sum[(prec, 0)] - 1.0
        g.close()
    out["edxct_paper"] = r

    # the EDXCT block made a scatterer (Sec. 3.3: the paper's phantom scatters
    # as it steps): water's energy-dependent Rayleigh and Compton tables, on
    # the 1/3-voxel march
    spec = wl.edxct_scatter_instrument()
    r = {}
    mons = [c for c, comp in enumerate(spec.components) if comp["type"].startswith("mon_")]
    for prec, n, kern in (("mixed", 50_000_000, "compiled"), ("mixed", 50_000_000, "generic"),
                          ("fp64", 5_000_000, "compiled")):
        g = mcx.Instrument(spec, precision=prec, device=dev, specialize=kern == "compiled")
        g.trace_range(0, n // 10, 4)
        g.reset()
        sec = timed(lambda: g.trace_range(10**10, 10**10 + n, 4))
        r[f"{prec}_{kern}"] = {"rays_per_s": n / sec, "rays": n,
                               "detected": int(sum(g.monitor(c)[0].sum() for c in mons)) / n}
        g.close()
    out["edxct_scattering_march3"] = r

    # the paper's focusing instrument (Sec. 3.2): Gaussian undulator source,
    # 16-lens Be CRL, 0.1 mm slit 14 m behind it, PSD and E monitor
    spec = wl.focusing_instrument()
    r = {}
    for prec, n, kern in (("mixed", 100_000_000, "compiled"), ("mixed", 100_000_000, "generic"),
                          ("fp64", 10_000_000, "compiled"), ("fp64", 10_000_000, "generic")):
        g = mcx.Instrument(spec, precision=prec, device=dev, specialize=kern == "compiled")
        g.trace_range(0, n // 10, 4)
        g.reset()
        sec = timed(lambda: g.trace_range(10**10, 10**10 + n, 4))
        r[f"{prec}_{kern}"] = {"rays_per_s": n / sec, "rays": n,
                               "through_slit": int(g.monitor(3)[0].sum()) / n}
        g.close()
    out["focusing_crl16"] = r

    # the paper's ray-count study (Sec. 5.1): the staircase test piece scanned
    # by 21 lines (ten through the lead rod, ten through steel alone, a flat
    # field) as one batch compiled by families; the CNR of the 26 mm step per
    # energy bin, its line fit above 80 keV and the criterion (fit > 1 over
    # 20-160 keV), for several rays per line; and the time a 550-line
    # projection at 1e7 rays per line takes at the measured rate
    import numpy as np
    from paper_2410_08747_gb300 import cnr as cnr_mod
    specs, labels = wl.staircase_scan()
    r = {}
    rate = None
    for n_line in (100_000, 1_000_000, 10_000_000):
        insts = [mcx.Instrument(s_, precision="mixed", device=dev) for s_ in specs]
        bs = mcx.Batch(insts, [n_line] * len(specs), chunk_rays=1 << 15)
        bs.specialize()
        bs.trace(30)                     # warm-up (graph capture), then cleared
        for i in insts:
            i.reset()
        sec = timed(lambda: bs.trace(31))
        sw = [i.monitor(4)[1].reshape(128, 128) for i in insts]
        st = cnr_mod.study(sw, labels, slice(59, 69))
        a, b_ = st["fit"]
        hi = st["cnr"][(st["e"] >= 80.0) & np.isfinite(st["cnr"])]
        r[f"{n_line:.0e}_rays_per_line"] = {
            "rays_per_s": n_line * len(specs) / sec, "seconds": sec,
            "cnr_fit_above_80keV": [a, b_] if math.isfinite(a) and math.isfinite(b_) else None,
            "passes": st["passes"],
            "cnr_median_above_80keV": float(np.median(hi)) if hi.size else None,
            "cnr_defined_bins": int(np.isfinite(st["cnr"]).sum())}
        rate = n_line * len(specs) / sec
        bs.close()
        for i in insts:
            i.close()
    r["projection_550_lines_1e7_seconds"] = 550 * 1e7 / rate
    out["edxct_staircase_cnr"] = r

    # batched: 360 rotated absorption projections + 16 slit instruments
    specs, budgets = wl.batched_workload()
    insts = [mcx.Instrument(s, precision="mixed", device=dev) for s in specs]
    b = mcx.Batch(insts, budgets)
    b.autotune(200_000)
    b.trace(1)
    sec_generic = timed(lambda: b.trace(2))
    # the kernel compiled by instrument families (compiled once, then tuned,
    # before timing)
    t0 = time.perf_counter()
    b.specialize()
    compile_s = time.perf_counter() - t0
    chosen = b.autotune(200_000)
    b.trace(1)
    sec = timed(lambda: b.trace(2))
    seq = timed(lambda: [i.trace_range(0, bud, 3) for i, bud in zip(insts, budgets)])
    out["batched_376"] = {"rays": int(sum(budgets)), "rays_per_s": sum(budgets) / sec,
                          "generic_kernel_rays_per_s": sum(budgets) / sec_generic,
                          "family_compile_seconds": compile_s,
                          "sequential_rays_per_s": sum(budgets) / seq, "launch": chosen,
                          "instruments": len(insts)}
    b.close()
    for i in insts:
        i.close()
    del insts

    out["learned_ct"] = learned_ct(mcx, wl, torch, dev, timed)
    return out


if __name__ == "__main__":
    main()
