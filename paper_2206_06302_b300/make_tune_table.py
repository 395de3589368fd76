"""Builds the tuner table shipped with the package (``tune_b300.json``).

Runs ``sx_tune`` (every candidate launch shape of the three kernel families, timed on scratch
arrays) for the four STREAM kernels in binary64 and binary32 at array sizes 2^lo .. 2^hi, then
``sx_tune_pass`` for each type and size (the four kernels timed together in a pass, which picks
the vector kernels' cache hints for that context), and writes the table with ``sx_tune_save``.
Entries the table already holds for this device are kept unless ``--retune``; the pass step runs
on every size unless ``--no-pass``.  Run it on the GPU model the table is for:

    python paper_2206_06302_b300/make_tune_table.py --lo 16 --hi 29
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import paper_2206_06302_b300 as sx  # noqa: E402

OPS = (("copy", sx.SX_OP_COPY), ("scale", sx.SX_OP_SCALE), ("add", sx.SX_OP_ADD), ("triad", sx.SX_OP_TRIAD))
TYPES = (("f64", sx.SX_F64), ("f32", sx.SX_F32))


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--lo", type=int, default=16, help="smallest log2 array size")
    ap.add_argument("--hi", type=int, default=29, help="largest log2 array size")
    ap.add_argument("--table", default=os.path.join(HERE, "tune_b300.json"), help="table to extend")
    ap.add_argument("--out", default="", help="where to write the table (default: --table)")
    ap.add_argument("--retune", action="store_true", help="tune entries the table already has")
    ap.add_argument("--no-pass", action="store_true", help="skip the pass tuner")
    a = ap.parse_args(argv)
    t = sx.sx_target_create(0)
    name = sx.sx_target_info_get(t)["name"]
    sx.sx_tune_clear()
    have = set()
    if os.path.exists(a.table):
        sx.sx_tune_load(a.table)
        with open(a.table) as f:
            have = {(e["op"], e["dtype"], e["bucket"]) for e in json.load(f).get("ops", []) if e["device"] == name}
    for b in range(a.lo, a.hi + 1):
        for tname, dt in TYPES:
            for oname, op in OPS:
                if (op, dt, b) in have and not a.retune:
                    continue
                t0 = time.perf_counter()
                cfg, gbs = sx.sx_tune(t, op, dt, 1 << b)
                print(json.dumps({"log2n": b, "dtype": tname, "op": oname, "GB/s": round(gbs, 1),
                                  "seconds": round(time.perf_counter() - t0, 2), "cfg": cfg}), flush=True)
            if not a.no_pass:
                t0 = time.perf_counter()
                cfgs, gbs = sx.sx_tune_pass(t, dt, 1 << b)
                print(json.dumps({"log2n": b, "dtype": tname, "pass GB/s": round(gbs, 1),
                                  "seconds": round(time.perf_counter() - t0, 2),
                                  "cache_hint": {oname: c["cache_hint"] for (oname, _), c in zip(OPS, cfgs)}}),
                      flush=True)
    sx.sx_tune_save(a.out or a.table)
    sx.sx_target_destroy(t)
    return 0


if __name__ == "__main__":
    sys.exit(main())
