"""Autotuner of the engine's shape-keyed partition (writes csrc/tuned.h).

The engine splits an instance's tiles into groups: a group is the unit of
its fixed-order reductions, so the number of groups must depend on the shape
alone (a problem solved alone and in a batch then sums in the same order and
gives the same bits).  How many groups one work item of a launch covers is
free: a lone solve takes one group per item (all the parallelism it has), a
crowded launch takes runs of groups.  This script measures, on the GPU it
runs on:

  * for lone solves of 2-D and 3-D grids over a range of sizes, the solve
    time with 1, 2 and 4 tiles per group (GPCG_GROUP_TILES), mixed
    precision at tau_rel 1e-6; the fastest per size becomes a range of the
    table (sizes are keyed by their number of 64 x 32 tiles);
  * for the 512-QP batch (a crowded launch whose shapes come from the same
    table), the batch time with the table restricted to at least 1, 2 and 4
    tiles per group: fine groups let a lone solve spread over more CTAs, but
    in a crowded launch each group end costs a block barrier and a
    reduction; the table keeps the finest lower bound whose batch time stays
    within 2 % of the coarsest one;
  * for that table, the batch time with 2, 4 and 8 tiles per work item
    (GPCG_ITEM_TILES).

It then writes the table (with the measurements as comments) to --out, by
default csrc/tuned.h; the library is rebuilt with it by _build.build().

    python -m paper_cs_0101018_gb300.tune [--out PATH]
"""
from __future__ import annotations

import argparse
import datetime
import json
import math
import os
import statistics
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GROUP_CANDIDATES = (1, 2, 4)
ITEM_CANDIDATES = (2, 4, 8)
SIDES_2D = (32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536)
SIDES_3D = (12, 16, 24, 32, 48, 64, 96, 128)
TX, TY = 64, 32


def n_tiles(dim: int, side: int) -> int:
    t = math.ceil(side / TX) * math.ceil(side / TY)
    return t * (side if dim == 3 else 1)


def _time_solve(g, qp, opts, reps: int = 5) -> float:
    import torch
    prob = g.gpcg_problem_create(qp)
    g.gpcg_solve(prob, opts)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.gpcg_solve(prob, opts)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def tune_groups(g, gi) -> list:
    """(dim, side, n_tiles, {G: ms}, best G) for each measured lone solve."""
    rows = []
    opts = g.default_options(tau_rel=1e-6, precision=g.MIXED, path=g.PATH_ENGINE)
    for dim, sides in ((2, SIDES_2D), (3, SIDES_3D)):
        for side in sides:
            qp = (gi.grid_qp_2d(side, side, seed=900 + side, shift=1e-2, bounds="two_sided")
                  if dim == 2 else
                  gi.grid_qp_3d(side, side, side, seed=900 + side, shift=1e-2, sigma=0.5,
                                bounds="two_sided", b_dist="uniform"))
            t = {}
            for gt in GROUP_CANDIDATES:
                os.environ["GPCG_GROUP_TILES"] = str(gt)
                t[gt] = _time_solve(g, qp, opts)
            os.environ.pop("GPCG_GROUP_TILES", None)
            best = min(GROUP_CANDIDATES, key=lambda k: (t[k], -k))
            rows.append((dim, side, n_tiles(dim, side), t, best))
            print(f"lone dim {dim} side {side}: " +
                  ", ".join(f"G={k} {v:.3f} ms" for k, v in t.items()), flush=True)
    return rows


def table_from(rows, g_min: int = 1) -> list:
    """Ranges of n_tiles with one group size each (the fastest lone solve
    among the sizes >= g_min): a measured size keys the range up to the
    geometric mid-point towards the next measured size."""
    out = []
    for dim in (2, 3):
        # sizes with the same number of tiles are one point (times summed)
        tot = {}
        for d, _, nt, t, _ in rows:
            if d == dim:
                acc = tot.setdefault(nt, {k: 0.0 for k in GROUP_CANDIDATES})
                for k in GROUP_CANDIDATES:
                    acc[k] += t[k]
        pts = sorted((nt, min((k for k in GROUP_CANDIDATES if k >= g_min),
                              key=lambda k: (t[k], -k)))
                     for nt, t in tot.items())
        lo = 1
        for k, (nt, best) in enumerate(pts):
            hi = (int(math.sqrt(nt * pts[k + 1][0])) if k + 1 < len(pts) else 1 << 30)
            if out and out[-1][0] == dim and out[-1][3] == best:
                out[-1] = (dim, out[-1][1], hi, best)
            else:
                out.append((dim, lo, hi, best))
            lo = hi + 1
    return out


def group_for(table, dim: int, nt: int) -> int:
    for d, lo, hi, gt in table:
        if d == dim and lo <= nt <= hi:
            return gt
    return 4


def _batch_ms(g, gi, table, item_tiles: int) -> float:
    """Best of 3 timed 512-QP batches (mixed, tau_rel 1e-6), the problems'
    groups from `table`."""
    import torch
    sides = gi.batch_sides()
    probs = []
    for k, s in enumerate(sides):
        os.environ["GPCG_GROUP_TILES"] = str(group_for(table, 2, n_tiles(2, int(s))))
        probs.append(g.gpcg_problem_create(gi.batch_instance(k, s)))
    os.environ.pop("GPCG_GROUP_TILES", None)
    os.environ["GPCG_ITEM_TILES"] = str(item_tiles)
    opts = g.default_options(tau_rel=1e-6, precision=g.MIXED)
    g.gpcg_solve_batch(probs, opts)
    ms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.gpcg_solve_batch(probs, opts)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    os.environ.pop("GPCG_ITEM_TILES", None)
    return min(ms)


def tune_floor(g, gi, rows, tolerance: float = 0.02) -> tuple:
    """The finest lower bound on the group size whose batch time stays within
    `tolerance` of the coarsest bound's; returns (g_min, {g_min: ms})."""
    ms = {}
    for g_min in sorted(GROUP_CANDIDATES, reverse=True):
        ms[g_min] = _batch_ms(g, gi, table_from(rows, g_min), 4)
        print(f"batch, groups of >= {g_min} tiles: {ms[g_min]:.1f} ms", flush=True)
    ref = ms[max(GROUP_CANDIDATES)]
    ok = [k for k in GROUP_CANDIDATES if ms[k] <= (1.0 + tolerance) * ref]
    return min(ok), ms


def tune_items(g, gi, table) -> dict:
    """Batch time of the 512-QP workload per tiles-per-item candidate."""
    out = {}
    for it in ITEM_CANDIDATES:
        out[it] = _batch_ms(g, gi, table, it)
        print(f"batch item tiles {it}: {out[it]:.1f} ms", flush=True)
    return out


def render(table, item_tiles: int, rows, items: dict, device: str, g_min: int,
           floors: dict, date: str = None) -> str:
    lines = [
        "// tuned.h -- the engine's shape-keyed partition, as measured by",
        "// paper_cs_0101018_gb300/tune.py (which rewrites this file).",
        "//",
        "// kTunedGroups: for grids of `dim` dimensions with n_tiles in [tiles_lo,",
        "// tiles_hi], the tiles per group (the reduction unit) that gave the fastest",
        "// lone solve among the sizes at least the floor the batch allows.",
        "// kTunedItemTiles: the tiles per work item of a launch with more groups",
        "// than the resident CTAs can take at once (batches, serving).",
        f"// Measured on {device}, {date or datetime.date.today().isoformat()}: mixed precision,",
        "// tau_rel 1e-6, median of 5 solves (ms) for 1 / 2 / 4 tiles per group:",
    ]
    for dim, side, nt, t, best in rows:
        lines.append(f"//   {dim}-D side {side:5d} ({nt:7d} tiles): " +
                     " / ".join(f"{t[k]:.3f}" for k in GROUP_CANDIDATES) +
                     f"  (fastest: {best})")
    lines.append("// 512-QP batch (best of 3, ms) with groups of at least " +
                 " / ".join(str(k) for k in sorted(floors)) + " tiles: " +
                 " / ".join(f"{floors[k]:.1f}" for k in sorted(floors)) +
                 f"  -> at least {g_min} (within 2 % of the coarsest)")
    lines.append("// 512-QP batch (best of 3, ms) for " +
                 " / ".join(str(k) for k in ITEM_CANDIDATES) + " tiles per item: " +
                 " / ".join(f"{items[k]:.1f}" for k in ITEM_CANDIDATES) + f"  -> {item_tiles}")
    lines += ["#pragma once", "", "namespace gpcg {", "", "struct TunedGroup {",
              "  int dim, tiles_lo, tiles_hi, group_tiles;", "};", "",
              "constexpr TunedGroup kTunedGroups[] = {"]
    for d, lo, hi, gt in table:
        hi_s = "1 << 30" if hi >= (1 << 30) else str(hi)
        lines.append(f"    {{{d}, {lo}, {hi_s}, {gt}}},")
    lines += ["};", f"constexpr int kTunedItemTiles = {item_tiles};", "", "}  // namespace gpcg", ""]
    return "\n".join(lines)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "csrc", "tuned.h"))
    ap.add_argument("--json", default=None, help="also write the measurements as JSON")
    ap.add_argument("--from-json", default=None,
                    help="write the table from the measurements of an earlier run's --json "
                         "instead of measuring")
    args = ap.parse_args()
    if args.from_json:
        with open(args.from_json) as f:
            d = json.load(f)
        rows = [(r["dim"], r["side"], r["n_tiles"], {int(k): v for k, v in r["ms"].items()},
                 r["best"]) for r in d["lone"]]
        floors = {int(k): v for k, v in d["batch_ms_by_floor"].items()}
        items = {int(k): v for k, v in d["batch_ms_by_item_tiles"].items()}
        g_min = int(d["group_floor"])
        table = table_from(rows, g_min)
        with open(args.out, "w") as f:
            f.write(render(table, int(d["item_tiles"]), rows, items, d["device"], g_min, floors,
                           d.get("date")))
        print("wrote", args.out)
        return
    import torch
    import gpcg_inputs as gi
    import paper_cs_0101018_gb300 as g
    g.load()
    device = torch.cuda.get_device_name(0)
    rows = tune_groups(g, gi)
    g_min, floors = tune_floor(g, gi, rows)
    table = table_from(rows, g_min)
    items = tune_items(g, gi, table)
    item_tiles = min(ITEM_CANDIDATES, key=lambda k: (items[k], k))
    with open(args.out, "w") as f:
        f.write(render(table, item_tiles, rows, items, device, g_min, floors))
    if args.json:
        with open(args.json, "w") as f:
            json.dump({"device": device, "date": datetime.date.today().isoformat(), "lone": [
                {"dim": d, "side": s, "n_tiles": nt, "ms": t, "best": b}
                for d, s, nt, t, b in rows], "batch_ms_by_floor": floors, "group_floor": g_min,
                "batch_ms_by_item_tiles": items, "table": table,
                "item_tiles": item_tiles}, f, indent=1)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
