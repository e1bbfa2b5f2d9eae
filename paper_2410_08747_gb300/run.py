"""Command-line runner for the synthetic instruments (the role McXtrace's
`mxrun` plays, Sec. 2.1): trace a named workload on one GPU and print the
throughput and a monitor summary as one JSON line.

    python -m paper_2410_08747_gb300.run --workload absorption --rays 1e7
    python -m paper_2410_08747_gb300.run --workload ct --rays 1e6 --precision fp64
    python -m paper_2410_08747_gb300.run --workload ct_window --rays 1e7 --learned --train 1e7
    python -m paper_2410_08747_gb300.run --workload absorption --rays 1e8 --compiled

Each run traces `--repeat` ranges of `--rays` rays (the first is a warm-up)
and reports the last one's CUDA-event time.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = ("flat", "absorption", "ct", "ct_window", "edxct", "edxct_march", "edxct_scatter",
             "focusing")


def build_spec(wl, name):
    if name == "flat":
        return wl.flat_slit_instrument()
    if name == "absorption":
        return wl.absorption_instrument()
    if name == "ct":
        return wl.ct_instrument()
    if name == "edxct":
        return wl.edxct_instrument()
    if name == "edxct_march":
        spec = wl.edxct_instrument()   # the paper's 1/3-voxel march
        spec.components[1]["march"] = 3
        return spec
    if name == "edxct_scatter":
        return wl.edxct_scatter_instrument()   # with water's scattering tables
    if name == "focusing":
        return wl.focusing_instrument()
    return wl.ct_instrument(window=1.5, spot=10e-6)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", choices=WORKLOADS, default="absorption")
    ap.add_argument("--rays", type=float, default=1e7)
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--compiled", action="store_true",
                    help="trace with the kernel compiled for this instrument")
    ap.add_argument("--learned", action="store_true",
                    help="draw ray starts from the learned proposal")
    ap.add_argument("--train", type=float, default=0,
                    help="with --learned: first train the proposal on this many plain-traced histories")
    ap.add_argument("--epochs", type=int, default=1)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=3e-3)
    args = ap.parse_args(argv)

    import torch

    from paper_2410_08747_gb300 import mcx
    from paper_2410_08747_gb300 import workloads as wl

    n = int(args.rays)
    spec = build_spec(wl, args.workload)
    inst = mcx.Instrument(spec, precision=args.precision, specialize=args.compiled)
    stream = torch.cuda.current_stream()
    prop = buf = None
    if args.learned:
        if args.precision != "mixed":
            ap.error("--learned needs --precision mixed")
        src = spec.components[0]
        mid, half = 0.5 * (src["e_min"] + src["e_max"]), 0.5 * (src["e_max"] - src["e_min"])
        prop = mcx.Proposal(0.1, 0.5 * src["target_w"], 0.5 * src["target_h"], [0, 0, mid, 0],
                            [1e5, 1e5, 1 / half, 1 / math.pi],
                            params=wl.proposal_init(0).astype("float32"))
        buf = torch.empty(6 * n, dtype=torch.float32, device="cuda")
        if args.train > 0:
            # histories: uniform starts traced by the same instrument, each with
            # the weight it left at the detector
            nh = int(args.train)
            hist = torch.empty(6 * nh, dtype=torch.float32, device="cuda")
            det = torch.empty(nh, dtype=torch.float32, device="cuda")
            trainer = mcx.Instrument(spec, precision="mixed", specialize=args.compiled)
            trainer.sample_starts(0, nh, args.seed + 1000, hist)
            trainer.trace_starts(hist, nh, 0, det)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            train_loss = prop.train(hist, det, nh, epochs=args.epochs, batch=args.batch, lr=args.lr)
            t1.record(stream)
            t1.synchronize()
            train_ms = t0.elapsed_time(t1)
            trainer.close()
            del hist, det
    ms = 0.0
    for r in range(max(1, args.repeat)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if prop is not None:
            prop.sample(inst, r * n, n, args.seed, buf)
            inst.trace_starts(buf, n, r * n)
        else:
            inst.trace_range(r * n, (r + 1) * n, args.seed)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
    out = {"workload": args.workload, "precision": args.precision, "compiled": bool(args.compiled),
           "learned": bool(args.learned),
           "rays": n, "ms": ms, "rays_per_s": n / (ms / 1e3)}
    mons = {}
    for c, comp in enumerate(spec.components):
        if comp["type"].startswith("mon_"):
            N, sw, _ = inst.monitor(c)
            mons[str(c)] = {"type": comp["type"], "counts": int(N.sum()), "sum_w": float(sw.sum())}
    out["monitors"] = mons
    if prop is not None and args.train > 0:
        out["training"] = {"histories": int(args.train), "epochs": args.epochs, "batch": args.batch,
                           "ms": train_ms, "last_loss": train_loss}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
