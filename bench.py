"""Benchmark: RF-CMP EFIE low-frequency sweep on a jittered level-5 geodesic sphere.

Workload (one step): a seeded, 3 %-jittered unit icosphere of frequency 32
(20480 cells, 30720 RWG unknowns); for ka = 1, 1e-1, ..., 1e-5 (a = 1 m): build
the operator (FP32 far-pair / FP64 near-pair assembly of T_A and V, the
dense (Sigma^T Sigma)^+ and G_ll^{-1} factors -- once per step, shared by the
six wavenumbers -- and alpha, beta, gamma by power iteration), excite it
with an x-polarised plane wave along +z, solve the RF-CMP system by
mixed-precision CG with float-float refinement to a relative residual of
1e-6, and evaluate the bistatic RCS on the E- and H-plane cuts (181 angles
each).  Metric: solves per second (6 solves per step), with per-solve
latency p50/p99.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (extrapolated to solves/s) on the host cores.  Multi-GPU runs are
independent replicas (one sweep per rank, no collective in the data path).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KA = [1.0, 1e-1, 1e-2, 1e-3, 1e-4, 1e-5]
TOL = 1e-6
WORKLOAD = "lowfreq_sweep_sphere_f32_n30720"
METRIC = "RF-CMP EFIE solves/s @1e-6 resid (ka sweep 1..1e-5, level-5 sphere)"
FP32_LANES_PER_SM = 128
N_SMS = 152
# DRAM traffic of a kernel family from one ncu capture of the current kernel, as the ratio of
# the captured dram__bytes_read.sum + dram__bytes_write.sum to the algorithmic bytes of that
# launch; the bench reports traffic per launch = ratio x its own algorithmic bytes per launch
# (traffic grows with the units, N^2).  Families without such a capture report None.
# gemv_c64_f32 (symmetric streaming kernel): 604.6 MB read + 4.0 MB written at N = 12000, two
# columns, against 4 N (N + 1) + 32 N x 2 = 576.8 MB (the tiles that cross the diagonal are read
# whole).  gemv_c64_ff (float-float streaming kernel, one column): 472.2 MB
# read + 3.3 MB written at N = 7680 against 8 N^2 + 32 N = 472.1 MB.
NCU_TRAFFIC_RATIO = {"gemv_c64_f32": (604.6 + 4.0) / 576.8, "gemv_c64_ff": (472.2 + 3.3) / 472.1}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


MESH_N = 32
MESH_KIND = "sphere"  # or "plate": the open square plate of MESH_N x MESH_N squares


def _mesh():
    import synth

    if MESH_KIND == "plate":
        return synth.plate(MESH_N, seed=7)
    return synth.geodesic_sphere(MESH_N, seed=2)


def _mesh_sizes():
    """(cells, unknowns) of the bench mesh."""
    n = MESH_N
    if MESH_KIND == "plate":
        return 2 * n * n, 3 * n * n - 2 * n
    return 20 * n * n, 30 * n * n


def _mesh_desc():
    c, u = _mesh_sizes()
    if MESH_KIND == "plate":
        return "open square plate %d x %d squares, %d cells, %d unknowns, jitter 3%%, seed 7" % (MESH_N, MESH_N, c, u)
    return "geodesic sphere frequency %d, %d cells, %d unknowns, jitter 3%%, seed 2" % (MESH_N, c, u)


def _cut_dirs():
    th = np.linspace(0.0, np.pi, 181)
    e = np.stack([np.sin(th), np.zeros_like(th), np.cos(th)], 1)
    h = np.stack([np.zeros_like(th), np.sin(th), np.cos(th)], 1)
    return np.concatenate([e, h])


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        # the raw samples stay on disk: $RFCMP_BENCH_OUT if set, else the temporary directory
        out = os.environ.get("RFCMP_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out, "clocks_bench_%d.csv" % device)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], p[5:9]):
                if v.lower() in ("active", "0x1") or v == "1":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device) -> float:
    """x reduced by MAX over the ranks of the default process group (x itself without one).

    Every rank runs its own replica of the workload (the path has no data exchange), so the job
    takes as long as its slowest rank.
    """
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world_size: int, ms_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world_size / (ms_max / 1e3)


def run_step(rf, ctx, mesh, dirs, kh, pol, lat, reports, tuning=None, host_io=None):
    """One pass of the hot path over the six wavenumbers; returns host bytes moved.

    host_io: None for device-resident vectors (the excitation is computed on the device, the
    currents stay there); else {ka: (e, j)} pinned host arrays of shape (1, N), and every solve
    goes through the C call with host buffers (rfcmp_solve_host: e copied in, j copied out),
    the far field then reading j uploaded again from the host."""
    import torch

    ctx.clear_cache()  # the topology factors are rebuilt once per step
    h2d = d2h = 0
    prev = None
    for ka in KA:
        t0 = time.perf_counter()
        # alpha, beta, gamma iterations start from the previous wavenumber's iterates
        op = rf.Operator(ctx, mesh.verts, mesh.tris, ka, scaling_start=prev)
        op.tuning = tuning
        if prev is not None:
            prev.close()
        h2d += mesh.verts.nbytes + mesh.tris.nbytes + dirs.nbytes
        if host_io is None:
            e = op.rhs_planewave(kh, pol)
            h2d += kh.nbytes + pol.nbytes
            j, rep = op.solve(e, tol=TOL)
        else:
            eh, jh = host_io[ka]
            _, rep = op.solve_host(eh, tol=TOL, out=jh)
            h2d += eh.nbytes
            d2h += jh.nbytes
            j = torch.from_numpy(jh).to("cuda", non_blocking=True)
            h2d += jh.nbytes
        rcs = op.farfield(j, dirs)
        d2h += rcs.nbytes
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - t0) * 1e3)
        reports.append((ka, rep[0], op.info()))
        prev = op
    if prev is not None:
        prev.close()
    return h2d, d2h


def host_excitations(rf, ctx, mesh, kh, pol):
    """{ka: (e, j)}: the plane-wave excitation of every wavenumber of the sweep in pinned host
    memory (the library's own rfcmp_rhs_planewave, computed once before any timing) and a pinned
    host buffer for the currents."""
    import torch

    out = {}
    for ka in KA:
        op = rf.Operator(ctx, mesh.verts, mesh.tris, ka, scaling="k")
        e = op.rhs_planewave(kh, pol)
        eh = torch.empty(e.shape, dtype=e.dtype, pin_memory=True)
        eh.copy_(e)
        jh = torch.empty(e.shape, dtype=e.dtype, pin_memory=True)
        out[ka] = (eh.numpy(), jh.numpy())
        op.close()
    torch.cuda.synchronize()
    return out


def _tuning(ctx, n, args):
    """The committed autotuner table of this device (None with --no-tuning or when absent)."""
    import torch

    from paper_1803_08333_gb300 import autotune

    if args.no_tuning:
        return None, "built-in"
    table = autotune.Table.for_device(torch.cuda.get_device_name(torch.cuda.current_device()))
    if table is None:
        return None, "built-in (no table for this device)"
    plan = table.lookup(n, 1, "mixed") or {}
    ctx.set_plan({"far_min_blocks": plan.get("far_min_blocks", 0)})
    return table, plan


def bench_ours(args):
    import torch

    import paper_1803_08333_gb300 as rf
    import synth
    from paper_1803_08333_gb300 import build

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    build.build()
    rf.set_solve_graphs(args.solve_graphs == "on")
    mesh = _mesh()
    dirs = _cut_dirs()
    kh, pol = synth.plane_wave_z()
    ctx = rf.Context(local)
    tuning, plan = _tuning(ctx, 3 * mesh.tris.shape[0] // 2, args)
    lat, reports = [], []
    for _ in range(args.warmup):
        run_step(rf, ctx, mesh, dirs, kh, pol, [], [], tuning=tuning)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(local)
    rf.profile_enable(True)
    barrier()
    launches0 = rf.launch_count()
    clocks.start()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        run_step(rf, ctx, mesh, dirs, kh, pol, lat, reports, tuning=tuning)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    gpu_launches = rf.launch_count() - launches0
    prof = rf.profile_read()
    rf.profile_enable(False)
    ms = max_over_ranks(ev0.elapsed_time(ev1), "cuda")
    solves = args.steps * len(KA) * ws
    value = job_rate(args.steps * len(KA), ws, ms)

    # end to end through the C calls with host buffers: host mesh in (rfcmp_op_create), host
    # excitation in and host currents out (rfcmp_solve_host), host RCS out (rfcmp_farfield)
    host_io = host_excitations(rf, ctx, mesh, kh, pol)
    e2e_lat = []
    barrier()
    t0 = time.perf_counter()
    h2d = d2h = 0
    for _ in range(args.steps):
        a, b = run_step(rf, ctx, mesh, dirs, kh, pol, e2e_lat, [], tuning=tuning, host_io=host_io)
        h2d += a
        d2h += b
    barrier()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, "cuda")

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return
    peaks, peak_kind = _peaks()
    roof, roof_more = roofline(prof, peaks, peak_kind, clk)
    total_kernel_ms = sum(v["total_ms"] for v in prof.values())
    kernels = {k: {"launches": v["launches"], "ms": round(v["total_ms"], 3),
                   "share_of_instrumented": round(v["total_ms"] / max(total_kernel_ms, 1e-9), 4)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["total_ms"])}
    iters = {("%g" % ka): r.iterations for ka, r, _ in reports[: len(KA)]}
    resid = max(r.residual for _, r, _ in reports)
    out = {
        "metric": METRIC,
        "value": round(value, 4),
        "unit": "solves/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 2),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "fp32 operator, float-float/fp64 refinement",
        "data": "synthetic (seeded jittered %s, plane wave)" % ("open plate" if MESH_KIND == "plate" else "icosphere"),
        "config": {
            "workload": WORKLOAD,
            "mesh": _mesh_desc(),
            "ka": KA,
            "tol": TOL,
            "nrhs": 1,
            "parallelism": "replicas" if ws > 1 else "single",
            "l2": "inputs larger than L2 (T_A complex64 %.2f GB, V %.2f GB)"
                  % (8e-9 * _mesh_sizes()[1] ** 2, 8e-9 * _mesh_sizes()[0] ** 2),
            "plan": plan,
            "solve_graphs": args.solve_graphs,
        },
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 2), "p99": round(float(np.percentile(lat, 99)), 2)},
        "iterations": iters,
        "max_residual": resid,
        "roofline": roof,
        "rooflines_next": roof_more,
        "kernels": kernels,
        "gpu_launches": gpu_launches,
        "clocks": clk,
        "e2e": {"value": round(solves / (e2e_ms / 1e3), 4), "unit": "solves/s", "h2d_bytes_per_step": int(h2d / args.steps),
                "d2h_bytes_per_step": int(d2h / args.steps)},
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_sample(args.cpu_budget)
    print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def _one_roofline(name, v, peaks, peak_kind, clk):
    avg_ms = v["total_ms"] / max(v["launches"], 1)
    if name.startswith("assemble_far"):
        mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = N_SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
        achieved = v["flops"] / v["launches"] / (avg_ms / 1e3) / 1e12
        return {"kernel": name, "bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                "flops_per_launch": v["flops"] / v["launches"], "avg_launch_ms": round(avg_ms, 4),
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x median SM clock"}
    if name.startswith("gemm_"):
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0)))
        achieved = v["flops"] / v["launches"] / (avg_ms / 1e3) / 1e12
        return {"kernel": name, "bound": "tensor", "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "flops_per_launch": v["flops"] / v["launches"], "avg_launch_ms": round(avg_ms, 4),
                "peak_source": "of %s bf16_tflops_sustained (issued BF16 MMA FLOPs: 3 split products for "
                               "gemm_bf16x3, 21 digit-pair products for gemm_exact)" % peak_kind}
    bytes_per = v["bytes"] / max(v["launches"], 1)
    achieved = bytes_per / (avg_ms / 1e3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    return {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": round(NCU_TRAFFIC_RATIO[name] * bytes_per) if name in NCU_TRAFFIC_RATIO else None,
            "bytes_per_launch": bytes_per, "avg_launch_ms": round(avg_ms, 4),
            "peak_source": "of %s hbm_gbs (MEASURED_PEAKS.json)" % peak_kind}


def roofline(prof, peaks, peak_kind, clk):
    """Roofline of the dominant kernel family with an algorithmic byte or FLOP count (and the next ones)."""
    rated = {k: v for k, v in prof.items() if (v["bytes"] > 0 or v["flops"] > 0) and v["launches"] > 0}
    if not rated:
        return None, []
    order = sorted(rated.items(), key=lambda kv: -kv[1]["total_ms"])
    rows = [_one_roofline(k, v, peaks, peak_kind, clk) for k, v in order[:4]]
    return rows[0], rows[1:]


def oracle_sample(budget_s: float = 20.0):
    """FP64 oracle on a bounded sample of the workload, extrapolated to solves/s.

    Sample: far+near moments of a few cell rows of the level-5 mesh at each ka
    (timed, scaled by N_C / rows to a full assembly of T_A and V), one dense
    complex128 matvec of 4096 x 4096 (scaled by entry count to the T_A, V,
    (Sigma^T Sigma)^+ and G_ll^{-1} products of one RF-CMP application), and a
    dense inverse of order 2048 (scaled by n^3 to the two factor inverses).
    Application count per solve: 3 x 30 power steps of 2 applications plus
    the CG iterations the oracle needs (23, its level-3 count) and a residual.
    """
    from oracle import efie

    mesh = _mesh()
    t_start = time.perf_counter()
    D = efie.discretize(mesh.verts, mesh.tris)
    t_disc = time.perf_counter() - t_start
    nc, N, nv = D.nc, D.N, D.nv
    rows = 24
    t_asm = 0.0
    for ka in KA:
        t0 = time.perf_counter()
        efie.pair_moments(D, np.arange(rows), ka)
        t_asm += (time.perf_counter() - t0) / rows * nc
        if time.perf_counter() - t_start > budget_s:
            break
    n = 4096
    rng = np.random.default_rng(0)
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    t0 = time.perf_counter()
    for _ in range(3):
        M @ x
    t_mv = (time.perf_counter() - t0) / 3 / (n * n)  # per complex entry
    B = rng.standard_normal((2048, 2048))
    B = B @ B.T + 2048 * np.eye(2048)
    t0 = time.perf_counter()
    np.linalg.inv(B)
    t_inv = (time.perf_counter() - t0) / 2048**3
    per_apply = t_mv * (2 * N * N + 2 * nc * nc + 4 * nc * nc * 0.5 + nv * nv * 0.5)
    applications = 3 * 30 * 2 / 2 + 23 + 2
    t_solves = len(KA) * applications * per_apply
    t_fact = t_inv * (nc**3 + nv**3)
    total = t_disc + t_asm / len(KA) * len(KA) + t_solves + t_fact
    cores = os.cpu_count()
    try:
        import threadpoolctl

        info = threadpoolctl.threadpool_info()
        cores = max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        pass
    return {
        "value": round(len(KA) / total, 6),
        "unit": "solves/s",
        "cores": cores,
        "kind": "oracle",
        "sample": "level-5 mesh: %d cell rows of pair moments per ka (x N_C/%d), one 4096^2 c128 matvec, one 2048^3 "
                  "inverse, extrapolated; %.1f s of CPU work" % (rows, rows, time.perf_counter() - t_start),
    }


def _scene_mesh(shape, n, cache):
    import synth

    key = (shape, n)
    if key not in cache:
        if shape == "sphere":
            cache[key] = synth.geodesic_sphere(n, seed=40 + n)
        elif shape == "ellipsoid":
            cache[key] = synth.ellipsoid(n, seed=40 + n)
        else:
            cache[key] = synth.cube(n, seed=40 + n)
    return cache[key]


def bench_serving(args):
    """Poisson stream of solves (seeded, 20 req/s) through the continuous-batching server.

    The 48 (mesh, ka) scenes of the pool are made resident first (operator assembly, scaling
    and the per-mesh factors; timed and reported as the cold phase), then the stream is
    replayed in real time against the warm server.
    """
    import threading

    import torch

    import synth
    from paper_1803_08333_gb300 import build, serve

    build.build()
    torch.cuda.set_device(0)
    work = serve.poisson_workload(args.requests, args.rate, seed=4, pool=args.scene_pool, mesh_pool=args.mesh_pool)
    meshes = {}
    scenes = [(_scene_mesh(sc[0], sc[1], meshes), sc[2], nr) for _, sc, nr in work]
    budget = int(torch.cuda.mem_get_info()[1] * 0.85)
    from paper_1803_08333_gb300 import autotune

    table = None if args.no_tuning else autotune.Table.for_device(torch.cuda.get_device_name(0))
    be = serve.GpuBackend(0, hbm_budget=0, tuning=table)
    srv = serve.Server(be, hbm_budget=budget, workers=args.workers, continuous=args.serve_mode == "continuous")
    t0 = time.perf_counter()
    seen = set()
    for _, sc, _ in work:
        if sc not in seen:
            seen.add(sc)
            m = _scene_mesh(sc[0], sc[1], meshes)
            srv.warm(m.verts, m.tris, sc[2])
    torch.cuda.synchronize()
    cold_s = time.perf_counter() - t0
    futs = [None] * len(work)

    def driver():
        t0 = time.perf_counter()
        for i, ((t_arr, _, _), (m, ka, nr)) in enumerate(zip(work, scenes)):
            delay = t_arr - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            kh, pol = synth.random_plane_waves(nr, seed=1000 + i)
            futs[i] = srv.submit(m.verts, m.tris, ka, kh, pol, tol=TOL)

    import paper_1803_08333_gb300 as rf

    clocks = Clocks(0)
    launches0 = rf.launch_count()
    clocks.start()
    th = threading.Thread(target=driver)
    t0 = time.perf_counter()
    th.start()
    th.join()
    res = [f.result() for f in futs]
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    gpu_launches = rf.launch_count() - launches0
    st = srv.stats()
    srv.close()
    sizes = sorted({3 * m.tris.shape[0] // 2 for m, _, _ in scenes})
    print(json.dumps({
        "metric": "RF-CMP EFIE serving: solves/s and p50/p99 latency @1e-6 resid", "value": st["solves_per_s"],
        "unit": "right-hand sides/s", "n_gpus": 1, "higher_is_better": True,
        "config": {"workload": f"poisson_serving_{args.rate:g}rps", "requests": args.requests, "scene_pool": len(seen),
                   "mesh_pool": len(meshes), "unknowns": [sizes[0], sizes[-1]], "workers": args.workers,
                   "budget_bytes": budget, "tol": TOL, "tuning": "table" if table is not None else "built-in",
                   "batching": args.serve_mode},
        "latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"]}, "requests_per_s": st["requests_per_s"],
        "queue_wait_ms": {"p50": st["p50_wait_ms"], "p99": st["p99_wait_ms"]}, "solves": st["solves"],
        "joined_running_solve": st["joined_running_solve"], "arrived_during_solve": st["arrived_during_solve"],
        "mean_batch_columns": st["mean_batch_columns"], "max_residual": max(max(r.residuals) for r in res),
        "resident_operators": st["resident_operators"], "cold_start_s": round(cold_s, 2), "wall_s": round(wall, 2),
        "gpu_launches": gpu_launches, "clocks": clk, "data": "synthetic (seeded jittered spheres, cubes, ellipsoids; random plane waves)"}))


def bench_batched(args):
    """512 plane waves on the 41070-unknown ellipsoid at ka = 2: one multi-column mixed solve per step.

    Beside it, the same right-hand sides one at a time in the float-float (FP64-equivalent)
    single-column form, on a sample of columns, for the batched-vs-single comparison.
    """
    import torch

    import paper_1803_08333_gb300 as rf
    import synth
    from paper_1803_08333_gb300 import autotune, build

    build.build()
    torch.cuda.set_device(0)
    nrhs, ka = args.nrhs, 2.0
    mesh = synth.ellipsoid(args.ellipsoid_n)  # semi-axes 1.0 / 0.6 / 0.4; n = 37: 27380 cells, 41070 unknowns
    kh, pol = synth.random_plane_waves(nrhs, seed=77)
    ctx = rf.Context(0)
    table = None if args.no_tuning else autotune.Table.for_device(torch.cuda.get_device_name(0))
    t0 = time.perf_counter()
    op = rf.Operator(ctx, mesh.verts, mesh.tris, ka)  # the major semi-axis is 1 m: k = ka
    op.tuning = table
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    e = op.rhs_planewave(kh, pol)
    for _ in range(args.warmup):
        op.solve(e, tol=TOL)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    rf.profile_enable(True)
    launches0 = rf.launch_count()
    clocks.start()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reps = []
    for _ in range(args.steps):
        j, rep = op.solve(e, tol=TOL)
        reps.append(rep)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    gpu_launches = rf.launch_count() - launches0
    prof = rf.profile_read()
    rf.profile_enable(False)
    ms = ev0.elapsed_time(ev1) / args.steps
    value = nrhs / (ms / 1e3)
    peaks, peak_kind = _peaks()
    roof, roof_more = roofline(prof, peaks, peak_kind, clk)
    # end to end: host right-hand sides in, host currents out, through the C call with host buffers
    eh = e.cpu().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    jh, _ = op.solve_host(eh, tol=TOL)
    e2e_s = time.perf_counter() - t0
    # the float-float single-column form on a sample of the columns
    single = []
    for c in range(args.single_sample):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, r1 = op.solve(e[c : c + 1], tol=TOL, precision="ff")
        torch.cuda.synchronize()
        single.append((time.perf_counter() - t0, r1[0]))
    single_s = float(np.median([t for t, _ in single]))
    last = reps[-1]
    print(json.dumps({
        "metric": "RF-CMP EFIE batched solves/s @1e-6 resid (512 plane waves, ellipsoid, ka=2)",
        "value": round(value, 3), "unit": "right-hand sides/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp32 operator; split-BF16 inner products; exact-digit residuals",
        "data": "synthetic (seeded jittered ellipsoid, seeded plane waves)",
        "config": {"workload": "batched_ellipsoid_n%d_rhs%d" % (op.N, nrhs), "unknowns": op.N, "ka": ka, "nrhs": nrhs,
                   "tol": TOL, "l2": "inputs larger than L2 (T_A complex64 13.5 GB)",
                   "tuning": "table" if table is not None else "built-in"},
        "setup_s": round(setup_s, 2),
        "iterations": [min(r.iterations for r in last), max(r.iterations for r in last)],
        "refinements": max(r.refinements for r in last),
        "max_residual": max(r.residual for r in last),
        "single_column_ff": {"solves_per_s": round(1.0 / single_s, 3), "sample_columns": args.single_sample,
                             "iterations": [r.iterations for _, r in single],
                             "max_residual": max(r.residual for _, r in single)},
        "batched_over_single": round(value * single_s, 1),
        "roofline": roof, "rooflines_next": roof_more, "gpu_launches": gpu_launches, "clocks": clk,
        "e2e": {"value": round(nrhs / e2e_s, 3), "unit": "right-hand sides/s",
                "h2d_bytes_per_step": int(eh.nbytes), "d2h_bytes_per_step": int(jh.nbytes)},
    }))


def bench_large(args):
    """The large instance: the seeded frequency-55 sphere (60500 cells, 90750 unknowns; T_A 65.9 GB
    of complex64), ka = 10 with 1024 seeded plane waves, then ka = 1e-4 with one plane wave, each
    solved by the mixed-precision RF-CMP CG with float-float refinement to 1e-6.

    The device memory is budgeted before anything is created: the resident operator (T_A, V and
    the two FP32 hi + lo factors), the BF16 planes the tensor-core inner products build, and the
    solve vectors of one block of columns must fit the free memory, which fixes the block of
    columns solved at once (512 on a GB300).  The six-digit exact planes of the accurate
    products would take 24 bytes per matrix entry (285 GB), so the accurate products stay on the
    float-float GEMV here (plan exact_min).
    """
    import torch

    import paper_1803_08333_gb300 as rf
    import synth
    from paper_1803_08333_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    n_geo = args.large_n
    mesh = synth.geodesic_sphere(n_geo, seed=5)
    nc = mesh.tris.shape[0]
    N, nv = 3 * nc // 2, nc // 2 + 2
    pad = lambda n: (n + 63) // 64 * 64  # noqa: E731
    op_bytes = 8 * (pad(N) * N + pad(nc) * nc) + 8 * (pad(nc) * nc + pad(nv) * nv)
    planes = 8 * (pad(N) * N + pad(nc) * nc) + 4 * (pad(nc) * nc + pad(nv) * nv)
    per_col = 16 * (14 * N + 10 * nc + 2 * nv) + 16 * 2 * N
    rf.pool_trim()
    free = torch.cuda.mem_get_info()[0]
    margin = 6 << 30
    cols = args.large_nrhs
    while cols > 4 and op_bytes + planes + per_col * cols + margin > free:
        cols //= 2
    if op_bytes + planes + per_col * cols + margin > free:
        raise SystemExit("large instance does not fit: %.1f GB free, %.1f GB needed"
                         % (free / 1e9, (op_bytes + planes + per_col * cols + margin) / 1e9))
    ctx = rf.Context(0)
    ctx.set_plan({"exact_min": 65536})
    rf.pool_reset_high()
    out = {"workload": "large_sphere_f%d_n%d" % (n_geo, N), "unknowns": N, "cells": nc,
           "budget": {"free_gb": round(free / 1e9, 1), "operator_gb": round(op_bytes / 1e9, 1),
                      "planes_gb": round(planes / 1e9, 1), "vectors_gb": round(per_col * cols / 1e9, 1),
                      "columns_per_solve": cols}}
    clocks = Clocks(0)
    clocks.start()
    for ka, nrhs in ((10.0, args.large_nrhs), (1e-4, 1)):
        t0 = time.perf_counter()
        op = rf.Operator(ctx, mesh.verts, mesh.tris, ka)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        info = op.info()
        kh, pol = synth.random_plane_waves(nrhs, seed=33) if nrhs > 1 else synth.plane_wave_z()
        t0 = time.perf_counter()
        reps = []
        for c0 in range(0, nrhs, cols):
            e = op.rhs_planewave(kh[c0 : c0 + cols], pol[c0 : c0 + cols])
            _, rep = op.solve(e, tol=TOL)
            reps += rep
            del e
        torch.cuda.synchronize()
        solve = time.perf_counter() - t0
        out["ka=%g" % ka] = {
            "nrhs": nrhs, "setup_s": round(setup, 2), "assembly_ms": round(info.ms_assembly, 1),
            "factors_ms": round(info.ms_factors, 1), "scaling_ms": round(info.ms_scaling, 1),
            "solve_s": round(solve, 2), "rhs_per_s": round(nrhs / solve, 2),
            "iterations": [min(r.iterations for r in reps), max(r.iterations for r in reps)],
            "refinements": max(r.refinements for r in reps), "converged": sum(r.converged for r in reps),
            "max_residual": max(r.residual for r in reps),
        }
        op.close()
    clk = clocks.stop()
    st = rf.pool_stats()
    out["memory_high_water_gb"] = {"used": round(st["used_high"] / 1e9, 1),
                                   "reserved": round(st["reserved_high"] / 1e9, 1)}
    out["clocks"] = clk
    print(json.dumps(out))


def bench_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    vals = []
    cb = None
    for _ in range(args.warmup + args.steps):
        cb = oracle_sample(args.cpu_budget)
        vals.append(cb["value"])
    v = float(np.median(vals[args.warmup:])) if args.steps > 0 else vals[-1]
    cb["value"] = v
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded jittered icosphere, plane wave)",
        "config": {"workload": WORKLOAD, "ka": KA, "tol": TOL, "nrhs": 1},
        "cpu_baseline": cb, "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mesh-n", type=int, default=32,
                    help="geodesic frequency of the sphere (32 = the workload; smaller for profiling captures)")
    ap.add_argument("--ka", type=float, nargs="*", default=None, help="override the wavenumber sweep")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "serving", "batched", "large"],
                    help="sweep: the level-5 low-frequency sweep (default); serving: the Poisson request stream; "
                         "batched: 512 plane waves on the 41070-unknown ellipsoid")
    ap.add_argument("--nrhs", type=int, default=512, help="batched: right-hand sides per solve")
    ap.add_argument("--ellipsoid-n", type=int, default=37,
                    help="batched: geodesic frequency of the ellipsoid (37 = the workload; smaller for profiling)")
    ap.add_argument("--single-sample", type=int, default=3, help="batched: columns solved one at a time in FF")
    ap.add_argument("--large-n", type=int, default=55,
                    help="large: geodesic frequency of the sphere (55 = 90750 unknowns)")
    ap.add_argument("--large-nrhs", type=int, default=1024, help="large: plane waves at ka = 10")
    ap.add_argument("--requests", type=int, default=600)
    ap.add_argument("--workers", type=int, default=4, help="serving: solver threads, one CUDA stream each")
    ap.add_argument("--serve-mode", default="continuous", choices=["continuous", "merged"],
                    help="serving: columns join running solves between sweeps, or merged solves run to the end")
    ap.add_argument("--rate", type=float, default=20.0, help="serving: mean arrivals per second")
    ap.add_argument("--scene-pool", type=int, default=48, help="serving: (mesh, ka) scenes the requests draw from")
    ap.add_argument("--mesh-pool", type=int, default=12, help="serving: meshes the scenes draw from")
    ap.add_argument("--no-tuning", action="store_true", help="ignore the autotuner table (built-in plans)")
    ap.add_argument("--mesh", default="sphere", choices=["sphere", "plate"],
                    help="sweep: the closed sphere (default) or an open square plate of --mesh-n squares a side "
                         "(give --mesh-n 100 for the 29800-unknown plate)")
    ap.add_argument("--solve-graphs", default="on", choices=["on", "off"],
                    help="sweep: solve loops as CUDA graphs (default), or the same kernels launched one by one "
                         "(every kernel then shows in a profiler's launch list)")
    args = ap.parse_args()
    global MESH_N, KA, WORKLOAD, METRIC, MESH_KIND
    if args.mesh == "plate":
        MESH_KIND = "plate"
        MESH_N = args.mesh_n
        KA = args.ka or KA
        WORKLOAD = "lowfreq_sweep_plate_n%d_N%d" % (MESH_N, _mesh_sizes()[1])
        METRIC = "RF-CMP EFIE solves/s @1e-6 resid (ka sweep 1..1e-5, open plate)"
    elif args.mesh_n != 32 or args.ka:
        MESH_N = args.mesh_n
        KA = args.ka or KA
        WORKLOAD = "profiling_case_sphere_f%d" % MESH_N
    if args.impl == "reference":
        bench_reference(args)
    elif args.workload == "serving":
        bench_serving(args)
    elif args.workload == "batched":
        bench_batched(args)
    elif args.workload == "large":
        bench_large(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
