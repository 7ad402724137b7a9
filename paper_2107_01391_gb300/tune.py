"""Tile-size tuner for the digit-group passes.

The library's pass kernel comes in two tile sizes for 4-byte cells: the wide
tile, fastest for large sorts, and a narrow one (16 keys per thread) that
spreads a sort of a few hundred thousand keys over more SMs.  Which is faster
depends on the device, so this module times both on the device at hand,
through the C ABI, and writes the crossover as a small JSON table:

    {"device_name": ..., "narrow_max_n": N, "measured": {...}}

``Context.apply_tuning(path)`` (or $RS_TUNE_FILE, read when the default
context is created) sets the context's limit from it; sorts of more than
4096 and at most N keys then take the narrow tile.  The result of a sort
does not depend on the tile.

    python -m paper_2107_01391_gb300.tune --out rs_tune.json
"""
from __future__ import annotations

import argparse
import json

DEFAULT_SIZES = tuple(1 << k for k in range(13, 24))
NEVER, ALWAYS = 0, 1 << 62


def crossover(times: dict[int, tuple[float, float]]) -> int:
    """The largest n such that the narrow tile is at least as fast as the wide
    one there and at every smaller measured n (times[n] = (wide_us,
    narrow_us)); 0 when the wide tile wins already at the smallest n."""
    best = 0
    for n in sorted(times):
        wide, narrow = times[n]
        if narrow > wide:
            break
        best = n
    return best


def measure(sizes=DEFAULT_SIZES, reps: int = 30, device: int = 0) -> dict:
    """Device time (us, CUDA events, mean of reps calls after warm-up) of the
    u32 pairs sort and the u32 keys sort at each n on both tiles."""
    import numpy as np
    import torch

    from . import binding, workloads as W

    torch.cuda.set_device(device)
    ctx = binding.Context(device)
    out = {"pairs": {}, "keys": {}}
    try:
        for n in sizes:
            k, v = W.u32_pairs(n, "uniform", seed_extra=n)
            dk = torch.from_numpy(k.view(np.int32)).cuda()
            dv = torch.from_numpy(v.view(np.int32)).cuda()
            ko, vo, o = torch.empty_like(dk), torch.empty_like(dv), torch.empty_like(dk)
            tp = torch.empty(binding.workspace_bytes("rs_sort_pairs_u32", n), dtype=torch.uint8,
                             device="cuda")
            tk = torch.empty(binding.workspace_bytes("rs_sort_u32", n), dtype=torch.uint8,
                             device="cuda")
            calls = {"pairs": lambda: binding.rs_sort_pairs(dk, dv, ko, vo, ctx=ctx, temp=tp),
                     "keys": lambda: binding.rs_sort_u32(dk, o, ctx=ctx, temp=tk)}
            for name, fn in calls.items():
                pair = []
                for limit in (NEVER, ALWAYS):
                    ctx.pass_tile_limit = limit
                    for _ in range(3):
                        fn()
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(reps):
                        fn()
                    e1.record()
                    torch.cuda.synchronize()
                    pair.append(e0.elapsed_time(e1) / reps * 1e3)
                out[name][n] = tuple(pair)
        ctx.check()
        name = torch.cuda.get_device_name(device)
    finally:
        ctx.close()
    return {"device_name": name, "times_us": out}


def table(measured: dict) -> dict:
    """The tuning table: the smaller of the two shapes' crossovers."""
    limit = min(crossover(measured["times_us"]["pairs"]), crossover(measured["times_us"]["keys"]))
    return {"device_name": measured["device_name"], "narrow_max_n": int(limit),
            "measured": {shape: {str(n): {"wide_us": round(w, 2), "narrow_us": round(nw, 2)}
                                 for n, (w, nw) in sorted(times.items())}
                         for shape, times in measured["times_us"].items()}}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default="rs_tune.json")
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--reps", type=int, default=30)
    ap.add_argument("--max-log2n", type=int, default=23)
    args = ap.parse_args(argv)
    sizes = tuple(1 << k for k in range(13, args.max_log2n + 1))
    t = table(measure(sizes, args.reps, args.device))
    with open(args.out, "w") as f:
        json.dump(t, f, indent=1)
        f.write("\n")
    print(json.dumps({"device_name": t["device_name"], "narrow_max_n": t["narrow_max_n"]}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
