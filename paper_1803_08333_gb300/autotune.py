"""Autotuner: launch shapes per (N, nrhs, precision), measured through the public API.

A plan (``paper_1803_08333_gb300.Plan``) fixes launch shapes only: the GEMV work-unit width
and persistent grid, the column count from which the inner-iteration products move from the
FP32 GEMV to the split-BF16 tensor-core GEMM, the GEMM N tile, and the register budget of the
far-pair assembly kernel.  None of them changes what a float-float product computes; the
inner-iteration products differ only by FP32 rounding order.

``tune_operator`` times candidates of one resident operator with CUDA events around
``rfcmp_apply`` (RFCMP_APPLY_A_INNER for MIXED solves: the operator application every inner CG
iteration performs; RFCMP_APPLY_A for FF) and keeps the fastest, one knob at a time
(coordinate descent from the built-in plan).  ``tune_assembly`` times operator creation.  The
results form a ``Table`` persisted as JSON and keyed by device name; ``Table.lookup`` returns the
plan of the nearest measured (N, nrhs) on a log scale, which ``Operator.solve`` applies when the
operator carries the table (``op.tuning = table``).

    python -m paper_1803_08333_gb300.autotune --out paper_1803_08333_gb300/tuning/<device>.json
"""

from __future__ import annotations

import argparse
import json
import math
import os
import re
from dataclasses import asdict, dataclass, field

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING_DIR = os.path.join(HERE, "tuning")

GEMV_CHUNKS = (256, 512, 1024, 2048, 4096)
GEMV_CTAS = (0, 1, 2, 4)
GEMM_BNS = (32, 64, 128)
FAR_MIN_BLOCKS = (1, 2, 3, 4)
# columns per call measured by default (the inner CG of a solve applies A to all active columns)
NRHS_GRID = (1, 2, 4, 8, 12, 16, 24, 32, 48, 64, 128, 256, 512)
GEMV_ONLY = 65536  # mrhs_min / exact_min that keeps every product on the GEMV
GEMM_ALWAYS = 1    # mrhs_min / exact_min that sends every multi-column product to the tensor cores


def device_slug(name: str) -> str:
    return re.sub(r"[^a-z0-9]+", "_", name.lower()).strip("_")


@dataclass
class Entry:
    n: int              # RWG unknowns of the operator measured
    nrhs: int           # columns per application
    precision: str      # "mixed" (inner iterations) or "ff"
    plan: dict          # Plan fields
    ms: float           # time of one application with this plan
    default_ms: float   # time with the built-in plan
    tried: dict = field(default_factory=dict)  # "knob=value" -> ms


class Table:
    """Tuned plans of one device."""

    def __init__(self, device: str, entries: "list[Entry] | None" = None):
        self.device = device
        self.entries: list[Entry] = list(entries or [])

    def add(self, e: Entry):
        self.entries = [x for x in self.entries if (x.n, x.nrhs, x.precision) != (e.n, e.nrhs, e.precision)]
        self.entries.append(e)

    def lookup(self, n: int, nrhs: int, precision: str = "mixed") -> "dict | None":
        """Plan of the nearest measured operator size, then the nearest column count (log scale)."""
        cands = [e for e in self.entries if e.precision == precision]
        if not cands or n <= 0 or nrhs <= 0:
            return None
        n_best = min({e.n for e in cands}, key=lambda m: (abs(math.log(m / n)), m))
        row = [e for e in cands if e.n == n_best]
        e = min(row, key=lambda x: (abs(math.log(x.nrhs / nrhs)), x.nrhs))
        return dict(e.plan)

    def to_json(self) -> dict:
        return {"device": self.device, "entries": [asdict(e) for e in self.entries]}

    @classmethod
    def from_json(cls, d: dict) -> "Table":
        return cls(d["device"], [Entry(**e) for e in d.get("entries", [])])

    def save(self, path: str):
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as f:
            json.dump(self.to_json(), f, indent=1, sort_keys=True)
            f.write("\n")

    @classmethod
    def load(cls, path: str) -> "Table":
        with open(path) as f:
            return cls.from_json(json.load(f))

    @classmethod
    def for_device(cls, name: str, directory: str = TUNING_DIR) -> "Table | None":
        """The committed table of a device, or None."""
        path = os.path.join(directory, device_slug(name) + ".json")
        if not os.path.exists(path):
            return None
        t = cls.load(path)
        return t if t.device == name else None


MIN_GAIN = 0.01  # a knob moves off its current value only for a gain above timing noise


def coordinate_descent(measure, knobs: "list[tuple[str, tuple]]", start: "dict | None" = None,
                       min_gain: float = MIN_GAIN):
    """Minimise measure(plan) over one knob at a time, in the given order.

    measure(plan dict) -> milliseconds (inf for an invalid candidate).  A candidate replaces the
    current plan only when it is faster by more than the fraction min_gain.  Returns
    (best plan, its ms, {"knob=value": ms} of every candidate tried).
    """
    plan = dict(start or {})
    best = measure(plan)
    tried = {"default": best}
    for name, values in knobs:
        for v in values:
            if plan.get(name, 0) == v:
                continue
            cand = dict(plan)
            cand[name] = v
            t = measure(cand)
            tried["%s=%d" % (name, v)] = t
            if t < best * (1.0 - min_gain):
                best, plan = t, cand
    return plan, best, tried


def _time_ms(fn, reps: int, warmup: int = 2) -> float:
    import torch

    for _ in range(warmup):
        fn()
    s = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
    times = []
    for i in range(reps):
        ev[2 * i].record(s)
        fn()
        ev[2 * i + 1].record(s)
    torch.cuda.synchronize()
    for i in range(reps):
        times.append(ev[2 * i].elapsed_time(ev[2 * i + 1]))
    times.sort()
    return times[len(times) // 2]


def tune_operator(op, nrhs_list=NRHS_GRID, precision: str = "mixed", reps: int = 5, seed: int = 0) -> "list[Entry]":
    """Tuned plans of one operator for each column count in nrhs_list."""
    import torch

    from . import RfcmpError

    which = "A_INNER" if precision == "mixed" else "A"
    g = torch.Generator(device="cpu").manual_seed(seed)
    out = []
    for nr in nrhs_list:
        x = torch.complex(torch.randn(nr, op.N, generator=g, dtype=torch.float64),
                          torch.randn(nr, op.N, generator=g, dtype=torch.float64)).cuda()
        y = torch.empty_like(x)

        def measure(plan, x=x, y=y):
            try:
                op.set_plan(plan)
                return _time_ms(lambda: op.apply(which, x, out=y), reps)
            except RfcmpError:
                return math.inf

        knobs = [("gemv_chunk", GEMV_CHUNKS), ("gemv_ctas_per_sm", GEMV_CTAS)]
        if precision == "mixed" and nr >= 2:
            knobs = [("mrhs_min", (GEMM_ALWAYS, GEMV_ONLY))] + knobs + [("gemm_bn", GEMM_BNS)]
        if precision == "ff" and nr >= 2:
            knobs = [("exact_min", (GEMM_ALWAYS, GEMV_ONLY))] + knobs
        default = measure({})
        plan, ms, tried = coordinate_descent(measure, knobs)
        if precision == "mixed" and plan.get("mrhs_min", 0) == GEMV_ONLY:
            plan.pop("gemm_bn", None)
        if plan:
            # the winner against the built-in plan once more, back to back: it must stay ahead
            ms, default = measure(plan), measure({})
            if ms >= default:
                plan, ms = {}, default
        out.append(Entry(op.N, nr, precision, plan, ms, default, tried))
        del x, y
    op.set_plan(None)
    return out


def tune_assembly(ctx, verts, tris, k: float, reps: int = 2) -> "tuple[int, dict]":
    """far_min_blocks with the fastest far-pair assembly of this mesh (scaling by k: no power steps)."""
    from . import Operator

    times = {}
    for b in FAR_MIN_BLOCKS:
        ctx.set_plan({"far_min_blocks": b})
        best = math.inf
        for _ in range(reps):
            op = Operator(ctx, verts, tris, k, scaling="k")
            best = min(best, float(op.info().ms_assembly))
            op.close()
        times[b] = best
    ctx.set_plan(None)
    return min(times, key=times.get), times


def main(argv=None):
    import torch

    import synth

    from . import Context, Operator, build

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", default=None, help="JSON table (default: tuning/<device>.json beside this file)")
    ap.add_argument("--sizes", type=int, nargs="*", default=[8, 16, 24, 32],
                    help="geodesic frequencies of the spheres tuned (30 n^2 unknowns each)")
    ap.add_argument("--nrhs", type=int, nargs="*", default=list(NRHS_GRID))
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args(argv)
    build.build()
    name = torch.cuda.get_device_name(0)
    out = args.out or os.path.join(TUNING_DIR, device_slug(name) + ".json")
    table = Table.load(out) if os.path.exists(out) else Table(name)
    ctx = Context(0)
    for n in args.sizes:
        m = synth.geodesic_sphere(n, seed=2)
        fmb, ftimes = tune_assembly(ctx, m.verts, m.tris, 1.0)
        op = Operator(ctx, m.verts, m.tris, 1.0)
        for prec, nrl in (("mixed", args.nrhs), ("ff", [1, 2, 4, 8, 16])):
            for e in tune_operator(op, nrl, prec, args.reps):
                e.plan["far_min_blocks"] = fmb
                e.tried.update({"far_min_blocks=%d" % b: t for b, t in ftimes.items()})
                table.add(e)
                print(json.dumps({"n": e.n, "nrhs": e.nrhs, "precision": e.precision, "plan": e.plan,
                                  "ms": round(e.ms, 4), "default_ms": round(e.default_ms, 4)}), flush=True)
        op.close()
        ctx.clear_cache()
    table.save(out)
    print("wrote", out)


if __name__ == "__main__":
    main()
