"""Measured peak rates of the hardware units the tracer's roofline divides by.

    python -m paper_2410_08747_gb300.peaks [--device D]

prints one JSON object: FFMA, IMAD and DFMA lane operations per second,
Philox4x32-10 blocks per second, and, over a sweep of array footprints,
monitor hits per second (three global atomic adds to one 24-byte bin at
random bins) and single u64 atomic adds per second (mcx_peak_measure).  The
footprint sweep shows where the atomic rate leaves L2.
"""

from __future__ import annotations

import argparse
import json

from . import mcx

FOOTPRINTS_MB = (4, 16, 32, 48, 64, 80, 100.663296, 128, 200, 400)


def measure(device: int = 0, footprints_mb=FOOTPRINTS_MB) -> dict:
    out = {k: mcx.peak_measure(k, device) for k in ("ffma", "imad", "philox", "dfma")}
    out["hit_per_s_by_mb"] = {}
    out["red_u64_per_s_by_mb"] = {}
    for mb in footprints_mb:
        fp = int(mb * 1e6) // 24 * 24
        out["hit_per_s_by_mb"][f"{mb:g}"] = mcx.peak_measure("hit", device, fp)
        out["red_u64_per_s_by_mb"][f"{mb:g}"] = mcx.peak_measure("red_u64", device, fp)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--device", type=int, default=0)
    args = ap.parse_args()
    print(json.dumps(measure(args.device), indent=1))


if __name__ == "__main__":
    main()
