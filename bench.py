"""Benchmark: the SPFD hot path on the 2 mm, ~9.25M-unknown body phantom.

One step is one pass of the whole hot path over the full-size workload
(256 x 160 x 896 voxels, h = 2 mm, 9,250,062 conducting nodes, loop source):
  spfd_build  -- edge conductances, unknowns, components, multigrid setup,
  spfd_solve  -- right-hand side, multigrid-preconditioned CG to a relative
                 residual of 1e-8, projection, Psi on the node grid,
  spfd_efield -- voxel-averaged |E|.
The headline line is the plain FP64 form; the mixed-precision form (FP64
refinement around an FP32/BF16 V-cycle CG) is timed on the same inputs and
reported beside it, and the adjoint gradient of J = mean |E|^2 (build +
solve + gradient on the 128 x 96 x 448 scaled body) in the "adjoint"
sub-object.  Inputs (3.7 GB working set) exceed the 129 MB L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank solves its own phantom copy (replicas: the
solve has no data-parallel split on one node in this design) and rank 0
prints the line.  ``--impl reference`` times the CPU FP64 oracle on the host
cores instead (rank 0 only).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2mm phantom solve time (s) to 1e-8 rel residual; stencil HBM GB/s vs peak; mixed vs FP64"
WORKLOAD = "body phantom 256x160x896 voxels, h=2 mm, 9,250,062 unknowns, loop source R=0.3 m, I=1000 A, 0.4 m below"
TOL = 1e-8
OMEGA = 2 * 3.141592653589793 * 85e3
# FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
GOLDEN = os.path.join(ROOT, "tests", "golden", "body_2mm_oracle.json")
DATA = "synthetic (seeded ellipsoid body phantom, 40 Voronoi tissues, analytic loop potential)"


def _config(world):
    """The workload, the same for both arms."""
    return {"workload": WORKLOAD, "tol": TOL, "precision": "fp64",
            "step": "build (edge conductances, unknowns, operator / preconditioner) + "
                    "solve of Eq. 3 to 1e-8 + voxel-averaged |E| (Eq. 1)",
            "l2": "inputs larger than L2 (3.7 GB device working set vs 129 MB L2)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": mx or None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist(backend="nccl"):
    """(rank, world, local rank, torch.distributed or None) from the torchrun
    environment; one process per GPU, each solving its own replica."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
        return rank, world, local, dist
    return 0, 1, local, None


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    if not dist:
        return float(x)
    import torch
    v = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return float(v.item())


def replica_value_s(step_ms_max, world):
    """Whole-job time per body: world replicas, one body each, finish in the
    slowest rank's step time."""
    return round(step_ms_max / 1000.0 / world, 6)


def _inputs():
    from spfd_inputs import body_phantom, loop_potential
    ph = body_phantom()
    a = loop_potential(ph.dims, ph.h, ph.origin)
    return ph, a


def pulled_nodes_of_a(sigma):
    """(rows, nodes) of a that spfd_pipeline_host reads from host memory: in
    each row (edge direction d, node row (j, k)) the nodes from the first
    conducting voxel of the voxel rows it touches to one past the last."""
    import numpy as np
    c = sigma > 0
    nz, ny, nx = c.shape
    anyr = c.any(axis=2)
    big = 1 << 30
    lo = np.where(anyr, c.argmax(axis=2), big)
    hi = np.where(anyr, nx - 1 - c[:, :, ::-1].argmax(axis=2) + 1, -1)
    L = np.full((nz + 2, ny + 2), big)
    H = np.full((nz + 2, ny + 2), -1)
    L[1:-1, 1:-1] = lo
    H[1:-1, 1:-1] = hi
    # node row (j, k) at [k + 1, j + 1]; its voxel rows are (j-1..j, k-1..k)
    def comb(views):
        lo_ = np.minimum.reduce([L[v] for v in views])
        hi_ = np.maximum.reduce([H[v] for v in views])
        return lo_, hi_
    v00, v01 = (slice(None, -1), slice(None, -1)), (slice(None, -1), slice(1, None))
    v10, v11 = (slice(1, None), slice(None, -1)), (slice(1, None), slice(1, None))
    rows = nodes = 0
    for lo_, hi_ in (comb([v00, v01, v10, v11]), comb([v01, v11]), comb([v10, v11])):
        ok = hi_ >= 0
        rows += int(ok.sum())
        nodes += int((hi_ - lo_ + 1)[ok].sum())
    return rows, nodes


def pushed_values_of_outputs(sigma):
    """Values of Psi and |E| that spfd_pipeline_host writes from the device
    into device-accessible host arrays (the host zeroes the rest): per node
    row the span of its unknowns, per voxel row the span of its conducting
    voxels."""
    import numpy as np
    c = sigma > 0
    nz, ny, nx = c.shape
    anyr = c.any(axis=2)
    imin = np.where(anyr, c.argmax(axis=2), -1)
    imax = np.where(anyr, nx - 1 - c[:, :, ::-1].argmax(axis=2), -1)
    n_e = int((imax - imin + 1)[anyr].sum())
    big = 1 << 30
    L = np.full((nz + 2, ny + 2), big)
    H = np.full((nz + 2, ny + 2), -1)
    L[1:-1, 1:-1] = np.where(anyr, imin, big)
    H[1:-1, 1:-1] = np.where(anyr, imax + 1, -1)
    lo = np.minimum.reduce([L[:-1, :-1], L[:-1, 1:], L[1:, :-1], L[1:, 1:]])
    hi = np.maximum.reduce([H[:-1, :-1], H[:-1, 1:], H[1:, :-1], H[1:, 1:]])
    ok = hi >= 0
    return int((hi - lo + 1)[ok].sum()), n_e


def oracle_errors(torch, psi, E):
    """Error of a GPU result against the CPU FP64 oracle's floor solution of
    the same workload (tests/golden/body_2mm_oracle.json, written from the
    oracle alone): relative L2 error of Psi over the 4096 seeded unknowns
    (both with zero mean per component) and the largest relative |E| error
    over the 8192 seeded conducting voxels, with the comparison floor
    1e-6 * max(max |E|, omega/h * max |a|)."""
    import numpy as np
    try:
        with open(GOLDEN) as f:
            g = json.load(f)
    except Exception:
        return None
    if "E_sample_voxels" not in g:
        return None
    dev = psi.device
    nodes = torch.tensor(g["psi_sample_nodes"], dtype=torch.int64, device=dev)
    vox = torch.tensor(g["E_sample_voxels"], dtype=torch.int64, device=dev)
    ps = psi.reshape(-1)[nodes].cpu().numpy()
    es = E.reshape(-1)[vox].cpu().numpy()
    pr = np.array(g["psi_sample_values"])
    er = np.array(g["E_sample_values"])
    floor = 1e-6 * max(g["E_max"], g["E_floor_scale"])
    return {"err_psi_vs_oracle": float(np.linalg.norm(ps - pr) / np.linalg.norm(pr)),
            "err_E_vs_oracle": float(np.max(np.abs(es - er) / np.maximum(er, floor))),
            "oracle_reference": f"oracle Jacobi-PCG floor solution (rel. residual "
                                f"{g['tol_1e-13']['rel_res']:.1e}); Psi at {len(pr)} seeded "
                                f"unknowns (relative L2), |E| at {len(er)} seeded conducting "
                                "voxels (max relative, floor 1e-6 of the field scale)"}


def run_ours(args):
    import numpy as np
    import torch

    import paper_2010_12879_gb300 as spfd

    rank, world, local, dist = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ph, a = _inputs()
    sig = torch.from_numpy(ph.sigma).to(dev)
    ad = torch.from_numpy(a).to(dev)
    stream = torch.cuda.current_stream(dev)
    nz, ny, nx = ph.sigma.shape
    psi = torch.empty((nz + 1, ny + 1, nx + 1), dtype=torch.float64, device=dev)
    E = torch.empty((nz, ny, nx), dtype=torch.float64, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()

    def one_step(precision, profile):
        opts = spfd.spfd_opts_default()
        opts.precision = precision
        opts.profile = 1 if profile else 0
        t = {}
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        S = spfd.Solver(sig, ph.h, opts, stream=stream)
        build_launches = S.info()["launches"]
        e[1].record(stream)
        _, info, st = S.solve(ad, TOL, psi)
        e[2].record(stream)
        S.efield(ad, psi, OMEGA, E)
        e[3].record(stream)
        torch.cuda.synchronize(dev)
        t["build_ms"] = e[0].elapsed_time(e[1])
        t["solve_ms"] = e[1].elapsed_time(e[2])
        t["efield_ms"] = e[2].elapsed_time(e[3])
        t["step_ms"] = e[0].elapsed_time(e[3])
        # kernels of this library launched in the step: build + solve + |E|
        t["launches"] = build_launches + info["launches"] + 1
        binfo = dict(info)
        stats = S.kernel_stats() if profile else []
        S.close()
        assert st == spfd.SPFD_OK and info["converged"], spfd.spfd_last_error()
        return t, binfo, stats

    def timed(precision, steps, warmup, profile):
        for _ in range(warmup):
            one_step(precision, profile)
        barrier()
        rec = []
        with ClockSampler(local) as clk:
            barrier()
            t0 = time.perf_counter()
            for _ in range(steps):
                rec.append(one_step(precision, profile))
            barrier()
            wall = time.perf_counter() - t0
        return rec, wall, clk.summary()

    hbm_peak, peak_kind = _peaks()
    K, W = args.steps, args.warmup
    # the FP64 pipe's rate on this GPU, measured by the library's probe
    # (independent FMA chains on every resident warp), beside the derived one
    try:
        fp64_measured, _ = spfd.spfd_fp64_fma_rate(stream.cuda_stream)
    except Exception:
        fp64_measured = None
    # timed steps run without per-launch events; the kernel table and the
    # roofline come from separate profiled steps (events around every launch)
    rec64, wall64, clk64 = timed(spfd.SPFD_FP64, K, W, False)
    err64 = oracle_errors(torch, psi, E)
    recmx, wallmx, clkmx = timed(spfd.SPFD_MIXED, K, W, False)
    errmx = oracle_errors(torch, psi, E)
    KP = max(1, min(K, 3))
    prof64 = [one_step(spfd.SPFD_FP64, True) for _ in range(KP)]
    profmx = [one_step(spfd.SPFD_MIXED, True) for _ in range(KP)]

    def agg(rec, prof):
        keys = rec[0][0].keys()
        out = {k: statistics.mean(r[0][k] for r in rec) for k in keys if rec[0][0][k] is not None}
        out["std_step_ms"] = statistics.pstdev(r[0]["step_ms"] for r in rec)
        info = rec[-1][1]
        fam = {}
        for r in prof:
            for s in r[2]:
                f = fam.setdefault(s["name"], {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0})
                for k in ("launches", "ms", "bytes", "flops"):
                    f[k] += s[k]
        return out, info, fam

    t64, info64, fam64 = agg(rec64, prof64)
    tmx, infomx, fammx = agg(recmx, profmx)

    # max over ranks of the mean step time
    step_ms = max_over_ranks(t64["step_ms"], dist, dev)

    def roofline(fam, kind):
        solve_fams = {k: v for k, v in fam.items() if not k.startswith("setup")}
        name, f = max(solve_fams.items(), key=lambda kv: kv[1]["ms"])
        per = f["ms"] / f["launches"]
        bytes_per = f["bytes"] / f["launches"]
        flops_per = f["flops"] / f["launches"]
        gbs = bytes_per / (per * 1e-3) / 1e9
        tfl = flops_per / (per * 1e-3) / 1e12
        # FP64 stencils sit above the machine balance of the FP64 pipe
        # (flop/byte > FP64 peak / HBM peak): bound by the FP64 ALU
        alu = name.endswith("_f64") and flops_per / max(bytes_per, 1) > FP64_PEAK_TFLOPS * 1e12 / (hbm_peak * 1e9)
        traffic = None
        tf = os.path.join(ROOT, "profiles", "ncu_traffic.json")
        if os.path.exists(tf):
            try:
                with open(tf) as fh:
                    traffic = json.load(fh).get(name)
            except Exception:
                traffic = None
        share = f["ms"] / sum(v["ms"] for v in solve_fams.values())
        if alu:
            return {"kernel": name, "bound": "alu", "achieved": round(tfl, 4),
                    "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                    "frac": round(tfl / FP64_PEAK_TFLOPS, 4), "traffic": traffic,
                    "peak_kind": "FP64 pipe, derived from unit counts and clocks",
                    "measured_fp64_fma_tflops": round(fp64_measured, 4) if fp64_measured else None,
                    "frac_of_measured": round(tfl / fp64_measured, 4) if fp64_measured else None,
                    "algorithmic_GBs": round(gbs, 1), "avg_launch_ms": round(per, 4),
                    "launches": f["launches"], "share_of_solve_kernel_time": round(share, 3)}
        return {"kernel": name, "bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(gbs / hbm_peak, 4), "traffic": traffic,
                "peak_kind": peak_kind, "avg_launch_ms": round(per, 4),
                "launches": f["launches"], "share_of_solve_kernel_time": round(share, 3)}

    roof64 = roofline(fam64, "fp64")
    roofmx = roofline(fammx, "mixed")

    # adjoint gradient: 128 x 96 x 448 voxels at 2 mm, the body's
    # ellipsoids scaled to the box, loop source; build + solve + gradient of
    # J = mean |E|^2 over conducting voxels, both solves to TOL
    adjoint = None
    if not args.no_adjoint:
        from spfd_inputs import loop_potential, scaled_body_phantom
        ph5 = scaled_body_phantom(128, 96, 448)
        a5 = torch.from_numpy(loop_potential(ph5.dims, ph5.h, ph5.origin)).to(dev)
        sig5 = torch.from_numpy(ph5.sigma).to(dev)
        recs = []
        for i in range(W + K):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(stream)
            S5 = spfd.Solver(sig5, ph5.h, stream=stream)
            e[1].record(stream)
            psi5, info5, st5 = S5.solve(a5, TOL)
            e[2].record(stream)
            J5, _, _, infoa, sta = S5.energy_grad(a5, psi5, OMEGA, TOL)
            e[3].record(stream)
            torch.cuda.synchronize(dev)
            S5.close()
            assert st5 == spfd.SPFD_OK and sta == spfd.SPFD_OK
            if i >= W:
                recs.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]),
                             e[2].elapsed_time(e[3]), e[0].elapsed_time(e[3])))
        mean = [statistics.mean(r[q] for r in recs) for q in range(4)]
        fd = adjoint_fd_check(spfd, torch, dev, stream, ph5, a5)
        adjoint = {"workload": "body phantom scaled to 128x96x448 voxels, h=2 mm, "
                               f"{info5['n_dof']} unknowns, loop source",
                   "objective": "J = mean over conducting voxels of |E|^2; dJ/dsigma per voxel, dJ/da per edge",
                   "tol": TOL, "ms_per_step": round(mean[3], 3),
                   "breakdown_ms": {"build_ms": round(mean[0], 3), "solve_ms": round(mean[1], 3),
                                    "grad_ms": round(mean[2], 3)},
                   "iters": info5["iters"], "adjoint_iters": infoa["iters"], "J": J5,
                   "check_vs_central_differences": fd}

    pct = None
    if not args.no_percentile:
        pct = bench_percentile(spfd, torch, dev, stream, ph, sig, ad, K, W)

    gauge = None
    if not args.no_tree_cotree:
        gauge = bench_tree_cotree(spfd, torch, dev, stream, ph, sig, ad, hbm_peak, peak_kind,
                                  K, W)

    cheb = None
    if not args.no_chebyshev:
        cheb = bench_chebyshev(spfd, torch, dev, stream, ph, sig, ad, psi, max(3, min(K, 5)), W)

    group = None
    if not args.no_group:
        group = bench_group(spfd, torch, dev, stream, ph, sig, ad, max(1, min(K, 5)), W)

    body1 = None
    if not args.no_1mm:
        body1 = bench_body_1mm(spfd, torch, dev, stream, 2, 1)

    batch = None
    if not args.no_batch:
        batch = bench_batch(spfd, torch, dev, stream, ph, sig, args.batch_rhs,
                            max(1, min(K, 3)), W)

    # end to end through the public API with host arrays: one
    # spfd_pipeline_host call per step (sigma and a in from pinned host
    # memory, Psi and |E| back to pinned host memory, every copy and kernel
    # inside the timed region)
    e2e = None
    if not args.no_e2e:
        sig_h = torch.from_numpy(ph.sigma).pin_memory()
        a_h = torch.from_numpy(a).pin_memory()
        psi_h = torch.empty(psi.shape, dtype=torch.float64).pin_memory()
        E_h = torch.empty(E.shape, dtype=torch.float64).pin_memory()
        times = []
        for i in range(W + K):
            barrier()
            t0 = time.perf_counter()
            st, pinfo = spfd.pipeline_host(sig_h, a_h, ph.h, TOL, OMEGA, psi_h, E_h,
                                           stream=stream.cuda_stream)
            dt = time.perf_counter() - t0
            assert st == spfd.SPFD_OK, spfd.spfd_last_error()
            if i >= W:
                times.append(dt)
        a_rows, a_nodes = pulled_nodes_of_a(ph.sigma)
        nx1 = ph.sigma.shape[2] + 1
        e2e = {"value": round(statistics.mean(times) / world, 6), "unit": "s",
               "value_kind": "host-to-host time of one body (s)" if world == 1 else
                             f"seconds per body over {world} replicas (time / {world})",
               "h2d_bytes_per_step": int(sig_h.numel() * 8 + a_nodes * 8),
               "d2h_bytes_per_step": int(8 * sum(pushed_values_of_outputs(ph.sigma))),
               "std_s": round(statistics.pstdev(times), 6),
               "median_s": round(statistics.median(times) / world, 6),
               "a_read": f"{a_nodes} nodes in {a_rows} of {3 * psi.shape[0] * psi.shape[1]} rows "
                         "of a (each row's span of edges of conducting voxels)",
               "iters": pinfo["iters"], "rel_res_true": pinfo["rel_res_true"],
               "path": "spfd_pipeline_host: pinned host sigma and a -> build, solve, |E| -> "
                       "pinned host Psi and |E|; sigma by the copy engine, the needed spans "
                       "of the rows of a pulled by SM loads during the build, the outputs "
                       "zeroed by host threads during the solve and their nonzero spans "
                       "written by SM stores after |E|; host wall clock per call"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(ph, a, iters=args.cpu_iters)

    if rank == 0:
        n_launch = int(round(t64["launches"] * K))
        line = {
            "metric": METRIC, "value": replica_value_s(step_ms, world), "unit": "s",
            "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": round(step_ms, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": DATA, "config": _config(world),
            "value_kind": ("step time of one body (s)" if world == 1 else
                           f"seconds per body: {world} replicas, one body each, finish in the "
                           f"slowest rank's step time; value = that time / {world} "
                           "(an inverse throughput), ms_per_step = the step latency"),
            "breakdown_ms": {k: round(v, 3) for k, v in t64.items()},
            "solve_s": round(t64["solve_ms"] / 1000.0, 6),
            "iters": info64["iters"], "rel_res_true": info64["rel_res_true"],
            "accuracy": err64,
            "n_dof": info64["n_dof"], "n_levels": info64["n_levels"],
            "mixed": {"ms_per_step": round(tmx["step_ms"], 3),
                      "solve_s": round(tmx["solve_ms"] / 1000.0, 6),
                      "breakdown_ms": {k: round(v, 3) for k, v in tmx.items()},
                      "iters": infomx["iters"], "outer_iters": infomx["outer_iters"],
                      "rel_res_true": infomx["rel_res_true"],
                      "accuracy": errmx,
                      "solve_speedup_vs_fp64": round(t64["solve_ms"] / tmx["solve_ms"], 3),
                      "step_speedup_vs_fp64": round(t64["step_ms"] / tmx["step_ms"], 3),
                      "roofline": roofmx, "clocks": clkmx},
            "roofline": roof64,
            "adjoint": adjoint,
            "percentile": pct,
            "tree_cotree": gauge,
            "chebyshev": cheb,
            "group": group,
            "body_1mm": body1,
            "batch": batch,
            "kernels_fp64": {k: {"launches": v["launches"] // KP, "ms": round(v["ms"] / KP, 4),
                                 "GBs": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1)}
                             for k, v in sorted(fam64.items(), key=lambda kv: -kv[1]["ms"])},
            "kernels_mixed": {k: {"launches": v["launches"] // KP, "ms": round(v["ms"] / KP, 4),
                                  "GBs": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1)}
                              for k, v in sorted(fammx.items(), key=lambda kv: -kv[1]["ms"])},
            "kernel_table": f"per-launch CUDA events over {KP} separate profiled steps per precision",
            "gpu_launches": n_launch,
            "clocks": clk64,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "timing": "CUDA events on the launch stream around each step, no per-launch events "
                      "inside the timed steps; kernel families from separate profiled steps",
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def bench_percentile(spfd, torch, dev, stream, ph, sig, ad, K, W):
    """Step 6 (Sec. II-A, Sec. III-E): the nearest-rank 99th percentile of
    the body's |E| per tissue (40 labels) and over the whole body, timed with
    CUDA events around spfd_percentile after W warm-up calls."""
    import numpy as np
    lab = torch.from_numpy(ph.labels.astype(np.int32)).to(dev)
    nlab = int(ph.tissue_sigma.size)
    with spfd.Solver(sig, ph.h, stream=stream, profile=1) as S:
        psi, info, st = S.solve(ad, TOL)
        E = S.efield(ad, psi, OMEGA)
        torch.cuda.synchronize(dev)
        S.kernel_stats(reset=True)
        rec = []
        for i in range(W + K):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            vals, cnts = S.percentile(E, lab, nlab, 0.99)
            e[1].record(stream)
            torch.cuda.synchronize(dev)
            if i == W - 1:
                S.kernel_stats(reset=True)
            if i >= W:
                rec.append(e[0].elapsed_time(e[1]))
        fam = [f for f in S.kernel_stats() if f["name"].startswith("percentile")]
    kms = sum(f["ms"] for f in fam) / K
    kbytes = sum(f["bytes"] for f in fam) / K
    return {"workload": "99th percentile (nearest rank) of the body's |E| per tissue (40 labels) "
                        "and over the whole body; |E| from the FP64 solve to 1e-8",
            "ms": round(statistics.mean(rec), 4), "kernel_ms": round(kms, 4),
            "launches": int(sum(f["launches"] for f in fam) // K),
            "algorithmic_GBs": round(kbytes / (kms * 1e-3) / 1e9, 1) if kms > 0 else None,
            "p99_body_V_per_m": vals[nlab], "conducting_voxels": int(cnts[nlab]),
            "p99_tissue_max_V_per_m": float(np.nanmax(vals[:nlab])),
            "timing": "CUDA events around the call (host round trips included); kernel_ms "
                      "sums the per-launch events of its kernels"}


def adjoint_fd_check(spfd, torch, dev, stream, ph, a, n_tissues=8, n_dirs=3, tol=1e-12):
    """The adjoint gradient of the adjoint workload against central
    differences of the GPU's own objective, every solve to `tol`: dJ/dsigma
    summed per tissue for a seeded subset of tissues (relative step 1e-6 of
    the tissue's conductivity), and dJ/da along seeded random directions (J is
    quadratic in a, so that difference is exact up to rounding).  Errors are
    normwise: the largest deviation over the tissues against the largest
    per-tissue gradient; per direction for dJ/da."""
    import numpy as np
    lab = ph.labels.astype(np.int64)
    air = lab < 0

    def sigma_of(table):
        s = np.asarray(table)[np.where(air, 0, lab)]
        s[air] = 0.0
        return torch.from_numpy(s).to(dev)

    def run(table, av, grads=False):
        with spfd.Solver(sigma_of(table), ph.h, stream=stream) as S:
            psi, _, st = S.solve(av, tol)
            J, dJda, dJds, info, st2 = S.energy_grad(av, psi, OMEGA, tol)
            assert st == spfd.SPFD_OK and st2 == spfd.SPFD_OK, spfd.spfd_last_error()
            return (J, dJda, dJds) if grads else J

    table = np.array(ph.tissue_sigma, dtype=np.float64)
    J0, dJda, dJds = run(table, a, grads=True)
    dJds = dJds.cpu().numpy()
    rng = np.random.default_rng(128)
    pick = np.sort(rng.choice(np.unique(lab[~air]), size=n_tissues, replace=False))
    adj = np.array([dJds[lab == t].sum() for t in pick])
    d = 1e-6
    fd = []
    for t in pick:
        tp, tm = table.copy(), table.copy()
        tp[t] *= 1 + d
        tm[t] *= 1 - d
        fd.append((run(tp, a) - run(tm, a)) / (2 * d * table[t]))
    err_s = float(np.abs(np.array(fd) - adj).max() / np.abs(adj).max())
    errs_a = []
    for _ in range(n_dirs):
        w = torch.from_numpy(rng.normal(size=tuple(a.shape))).to(dev)
        eps = 1e-3 * float(a.abs().max()) / float(w.abs().max())
        fd_a = (run(table, a + eps * w) - run(table, a - eps * w)) / (2 * eps)
        an = float((dJda * w).sum())
        errs_a.append(abs(fd_a - an) / abs(an))
    return {"tol": tol, "tissues": [int(t) for t in pick], "relative_step": d,
            "max_rel_err_dJdsigma_per_tissue": err_s,
            "max_rel_err_dJda_directional": float(max(errs_a)),
            "directions": n_dirs}


def bench_chebyshev(spfd, torch, dev, stream, ph, sig, ad, psi, K, W):
    """The V-cycle's smoother: weighted Jacobi V(1,1) (the default) against
    Chebyshev of degree 2 and 3 (fused residual-and-update sweeps) on the
    2 mm body, FP64 and mixed, solve to TOL: median solve time over K solves
    after W warm-up solves on one built context each (CUDA events on the
    stream), iterations and the true residual."""
    out = {"workload": "2 mm body, loop source, solve to 1e-8 (build excluded)", "runs": []}
    for prec, pname in ((spfd.SPFD_FP64, "fp64"), (spfd.SPFD_MIXED, "mixed")):
        for sm, deg in ((spfd.SPFD_SMOOTHER_JACOBI, 0), (spfd.SPFD_SMOOTHER_CHEBYSHEV, 2),
                        (spfd.SPFD_SMOOTHER_CHEBYSHEV, 3)):
            opts = spfd.spfd_opts_default()
            opts.precision = prec
            opts.smoother = sm
            if deg:
                opts.cheb_degree = deg
            times = []
            with spfd.Solver(sig, ph.h, opts, stream=stream) as S:
                for i in range(W + K):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    _, info, st = S.solve(ad, TOL, psi)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    assert st == spfd.SPFD_OK, spfd.spfd_last_error()
                    if i >= W:
                        times.append(e0.elapsed_time(e1))
            out["runs"].append({"precision": pname,
                                "smoother": "jacobi V(1,1)" if not deg else f"chebyshev degree {deg}",
                                "solve_ms": round(statistics.median(times), 3),
                                "iters": info["iters"], "outer_iters": info["outer_iters"],
                                "rel_res_true": info["rel_res_true"]})
    return out


def bench_tree_cotree(spfd, torch, dev, stream, ph, sig, ad, hbm_peak, peak_kind, K, W):
    """Step 3 (Sec. II-A, Eq. 2): edge potentials from facet fluxes by
    tree-cotree gauging (comb tree on the grid's central root line) on the
    2 mm body grid.  The fluxes are the loop's closed-form B integrated over
    every facet (4 x 4 Gauss-Legendre, made on the device).  Times the gauge
    kernel alone (CUDA events, W warm-up launches, inputs and outputs of
    890 MB each, larger than L2), then steps 3-5 (gauge + build + solve to
    TOL + |E|), and compares |E| with the one of the loop's midpoint-sampled
    potentials (the headline's source: the same field discretised another
    way, O(h^2) apart)."""
    import numpy as np

    from spfd_inputs.sources_torch import loop_flux_t
    nz, ny, nx = ph.sigma.shape
    t0 = time.perf_counter()
    b = loop_flux_t(ph.dims, ph.h, ph.origin, order=4, device=dev)
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    ap = torch.empty_like(b)
    j0, k0 = ny // 2, nz // 2
    NN = (nx + 1) * (ny + 1) * (nz + 1)
    rec = []
    for i in range(W + K):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        spfd.spfd_tree_cotree(b.data_ptr(), nx, ny, nz, j0, k0, stream.cuda_stream,
                              ap.data_ptr())
        e[1].record(stream)
        torch.cuda.synchronize(dev)
        if i >= W:
            rec.append(e[0].elapsed_time(e[1]))
    ms = statistics.mean(rec)
    gbs = 40.0 * NN / (ms * 1e-3) / 1e9
    psi = torch.empty((nz + 1, ny + 1, nx + 1), dtype=torch.float64, device=dev)
    E = torch.empty((nz, ny, nx), dtype=torch.float64, device=dev)
    steps = []
    for i in range(W + K):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        e[0].record(stream)
        spfd.spfd_tree_cotree(b.data_ptr(), nx, ny, nz, j0, k0, stream.cuda_stream,
                              ap.data_ptr())
        e[1].record(stream)
        S = spfd.Solver(sig, ph.h, stream=stream)
        e[2].record(stream)
        _, info, st = S.solve(ap, TOL, psi)
        e[3].record(stream)
        S.efield(ap, psi, OMEGA, E)
        e[4].record(stream)
        torch.cuda.synchronize(dev)
        S.close()
        assert st == spfd.SPFD_OK, spfd.spfd_last_error()
        if i >= W:
            steps.append([e[q].elapsed_time(e[q + 1]) for q in range(4)] +
                         [e[0].elapsed_time(e[4])])
    m = [statistics.mean(r[q] for r in steps) for q in range(5)]
    # |E| of the midpoint-sampled potentials at the same tolerance
    with spfd.Solver(sig, ph.h, stream=stream) as S:
        psi_m, info_m, _ = S.solve(ad, TOL)
        E_m = S.efield(ad, psi_m, OMEGA)
    mask = torch.from_numpy(ph.sigma > 0).to(dev)
    Emax = float(E_m[mask].max())
    rel = (E - E_m).abs()[mask] / torch.clamp(E_m[mask], min=1e-6 * Emax)
    out = {"workload": "facet fluxes of the loop (R=0.3 m, I=1000 A, 0.4 m below) on the "
                       "256x160x896 grid (37.1 M nodes, 111 M facets), 4x4 Gauss-Legendre per "
                       "facet; comb tree on the central root line",
           "kernel_ms": round(ms, 4), "launches": 1,
           "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak,
                        "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
                        "peak_kind": peak_kind,
                        "algorithmic_bytes": "40 per node (read b_x, b_y; write a_x, a_y, a_z)"},
           "steps_3_to_5_ms": round(m[4], 3),
           "breakdown_ms": {"tree_cotree": round(m[0], 3), "build": round(m[1], 3),
                            "solve": round(m[2], 3), "efield": round(m[3], 3)},
           "iters": info["iters"], "iters_midpoint_source": info_m["iters"],
           "rel_res_true": info["rel_res_true"],
           "E_max_rel_diff_vs_midpoint_source": float(rel.max()),
           "E_p99_V_per_m": float(torch.quantile(E[mask][::64], 0.99)),
           "flux_generation_s": round(gen_s, 2), "steps": K, "warmup": W}
    del b, ap, psi, E, psi_m, E_m
    torch.cuda.empty_cache()
    return out


def uneven_phantom_dims(n=12):
    """n box sizes from 64x64x128 to 192x128x640 voxels, each axis
    interpolated linearly and rounded to a multiple of 32."""
    out = []
    for i in range(n):
        t = i / (n - 1)
        out.append(tuple(int(round((lo + t * (hi - lo)) / 32.0)) * 32
                         for lo, hi in ((64, 192), (64, 128), (128, 640))))
    return out


def bench_body_1mm(spfd, torch, dev, stream, K, W):
    """The second workload: the same ellipsoid body at h = 1 mm (512 x 320 x
    1792 voxels, 71.6 M conducting voxels, ~74 M unknowns), the same 40
    seeded tissues and loop source, on one GPU.  Per precision, W + K steps
    of build + solve to TOL + |E| + the per-tissue 99th percentile, each
    timed with CUDA events on the stream.  The loop's edge potentials are
    generated on the device."""
    import numpy as np

    from spfd_inputs import body_phantom
    from spfd_inputs.sources_torch import loop_potential_t
    t0 = time.perf_counter()
    ph = body_phantom(512, 320, 1792, h=1e-3)
    gen_s = time.perf_counter() - t0
    sig = torch.from_numpy(ph.sigma).to(dev)
    lab = torch.from_numpy(ph.labels.astype(np.int32)).to(dev)
    nlab = int(ph.tissue_sigma.size)
    a = loop_potential_t(ph.dims, ph.h, ph.origin, device=dev)
    nz, ny, nx = ph.sigma.shape
    psi = torch.empty((nz + 1, ny + 1, nx + 1), dtype=torch.float64, device=dev)
    E = torch.empty((nz, ny, nx), dtype=torch.float64, device=dev)
    out = {"workload": "body phantom 512x320x1792 voxels, h=1 mm, 40 tissues, loop source "
                       "R=0.3 m, I=1000 A, 0.4 m below; FP64 / mixed to 1e-8",
           "conducting_voxels": int((ph.sigma > 0).sum()),
           "phantom_generation_s_host": round(gen_s, 1), "steps": K, "warmup": W}
    for name, prec in (("fp64", spfd.SPFD_FP64), ("mixed", spfd.SPFD_MIXED)):
        rec = []
        for i in range(W + K):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            e[0].record(stream)
            S = spfd.Solver(sig, ph.h, stream=stream, precision=prec)
            e[1].record(stream)
            _, info, st = S.solve(a, TOL, psi)
            e[2].record(stream)
            S.efield(a, psi, OMEGA, E)
            e[3].record(stream)
            vals, _ = S.percentile(E, lab, nlab, 0.99)
            e[4].record(stream)
            torch.cuda.synchronize(dev)
            bi = S.info()
            S.close()
            assert st == spfd.SPFD_OK and info["converged"], spfd.spfd_last_error()
            if i >= W:
                rec.append([e[q].elapsed_time(e[q + 1]) for q in range(4)] +
                           [e[0].elapsed_time(e[4])])
        m = [statistics.mean(r[q] for r in rec) for q in range(5)]
        out[name] = {"build_ms": round(m[0], 2), "solve_ms": round(m[1], 2),
                     "efield_ms": round(m[2], 2), "percentile_ms": round(m[3], 2),
                     "step_ms": round(m[4], 2), "iters": info["iters"],
                     "outer_iters": info["outer_iters"], "rel_res_true": info["rel_res_true"],
                     "n_dof": int(bi["n_dof"]), "n_levels": int(bi["n_levels"]),
                     "context_bytes_device": int(bi["bytes_device"]),
                     "p99_body_V_per_m": vals[nlab]}
    del sig, lab, a, psi, E
    torch.cuda.empty_cache()
    return out


def bench_group(spfd, torch, dev, stream, ph, sig, ad, K, W):
    """Several bodies at once (multi-phantom workload): 12 ellipsoid bodies
    scaled to boxes from 64x64x128 to 192x128x640 voxels (h = 2 mm, tissues
    seeded as for the 2 mm body), one loop source each, solved to TOL
    (a) one after the other with spfd_solve and (b) together by one launch of
    the group's captured graph (spfd_group_solve), in FP64 and in the mixed
    form; plus the 2 mm body alone, host-driven against its captured graph.
    CUDA events on the stream."""
    from spfd_inputs import loop_potential, scaled_body_phantom
    dims = uneven_phantom_dims()
    phs = [scaled_body_phantom(*d) for d in dims]
    sigs = [torch.from_numpy(p.sigma).to(dev) for p in phs]
    A = [torch.from_numpy(loop_potential(p.dims, p.h, p.origin)).to(dev) for p in phs]
    solvers = [spfd.Solver(s, p.h, stream=stream) for s, p in zip(sigs, phs)]
    psis = [torch.empty(S.node_shape, dtype=torch.float64, device=dev) for S in solvers]

    def timed(fn, k, w):
        for _ in range(w):
            fn()
        rec = []
        for _ in range(k):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            out = fn()
            e[1].record(stream)
            torch.cuda.synchronize(dev)
            rec.append(e[0].elapsed_time(e[1]))
        return statistics.mean(rec), out

    def seq_and_group(solvers):
        def sequential():
            infos = []
            for S, a, p in zip(solvers, A, psis):
                _, info, st = S.solve(a, TOL, p)
                assert st == spfd.SPFD_OK, spfd.spfd_last_error()
                infos.append(info)
            return infos
        ms_seq, infos_seq = timed(sequential, K, W)
        ref = [p.clone() for p in psis]
        with spfd.Group(solvers, stream=stream) as G:
            def grouped():
                _, infos, st = G.solve(A, TOL, psis)
                assert st == spfd.SPFD_OK, spfd.spfd_last_error()
                return infos
            t0 = time.perf_counter()
            grouped()  # captures and instantiates the graph
            capture_ms = (time.perf_counter() - t0) * 1e3
            ms_grp, infos_grp = timed(grouped, K, W)
            same = all(torch.equal(a, b) for a, b in zip(ref, psis))
        return ms_seq, infos_seq, ms_grp, infos_grp, capture_ms, same

    try:
        ms_seq, infos_seq, ms_grp, infos_grp, capture_ms, same = seq_and_group(solvers)
        for S in solvers:
            S.close()
        solvers = [spfd.Solver(s, p.h, stream=stream, precision=spfd.SPFD_MIXED)
                   for s, p in zip(sigs, phs)]
        mx = seq_and_group(solvers)
        # the 2 mm body alone: host-driven solve against its captured graph
        psi_b = torch.empty((ph.sigma.shape[0] + 1, ph.sigma.shape[1] + 1,
                             ph.sigma.shape[2] + 1), dtype=torch.float64, device=dev)
        with spfd.Solver(sig, ph.h, stream=stream) as SB:
            ms_bh, ib = timed(lambda: SB.solve(ad, TOL, psi_b)[1], K, W)
            with spfd.Group([SB], stream=stream) as GB:
                ms_bg, ibg = timed(lambda: GB.solve([ad], TOL, [psi_b])[1][0], K, W)
    finally:
        for S in solvers:
            S.close()
    return {"workload": "12 ellipsoid bodies scaled to boxes from 64x64x128 to 192x128x640 "
                        "voxels (h=2 mm, 40 seeded tissues), one loop source each, FP64 to 1e-8",
            "dims": [list(d) for d in dims],
            "unknowns": [int(i["n_dof"]) for i in infos_seq],
            "iters": [int(i["iters"]) for i in infos_grp],
            "sequential_ms": round(ms_seq, 3), "group_graph_ms": round(ms_grp, 3),
            "speedup_group_vs_sequential": round(ms_seq / ms_grp, 3),
            "group_capture_ms": round(capture_ms, 1),
            "graph_launches_per_group_solve": 1,
            "kernels_in_graph": int(infos_grp[0]["launches"]),
            "bit_identical_to_sequential": bool(same),
            "mixed": {"sequential_ms": round(mx[0], 3), "group_graph_ms": round(mx[2], 3),
                      "speedup_group_vs_sequential": round(mx[0] / mx[2], 3),
                      "group_capture_ms": round(mx[4], 1),
                      "iters": [int(i["iters"]) for i in mx[3]],
                      "outer_iters": [int(i["outer_iters"]) for i in mx[3]],
                      "bit_identical_to_sequential": bool(mx[5]),
                      "group_mixed_vs_group_fp64": round(ms_grp / mx[2], 3)},
            "body_2mm": {"host_driven_solve_ms": round(ms_bh, 3),
                         "graph_solve_ms": round(ms_bg, 3),
                         "iters": int(ibg["iters"]), "rel_res_true": ibg["rel_res_true"]},
            "steps": K, "warmup": W}


def bench_batch(spfd, torch, dev, stream, ph, sig, nrhs, K, W):
    """Many source fields on one body (batched-source workload): nrhs loops
    at seeded positions (x, y in +-0.5 m, z in -0.6..-0.3 m) and random
    orientations, made on the device.  For each precision (plain FP64 and
    the mixed form), one context solves all fields to TOL as one
    spfd_solve_batch call and as nrhs spfd_solve calls, each timed with CUDA
    events on the context's stream after W warm-up rounds."""
    import numpy as np

    from spfd_inputs import random_loops
    from spfd_inputs.sources_torch import loop_potential_t
    loops = random_loops(nrhs, np.random.default_rng(4))
    nshape = tuple(d + 1 for d in ph.dims[::-1])
    A = torch.empty((nrhs, 3) + nshape, dtype=torch.float64, device=dev)
    for j, (c, n) in enumerate(loops):
        loop_potential_t(ph.dims, ph.h, ph.origin, center=c, normal=n, device=dev, out=A[j])
    psi = torch.empty((nrhs,) + nshape, dtype=torch.float64, device=dev)

    def run(precision, autotune=1, sequential_too=True):
        S = spfd.Solver(sig, ph.h, stream=stream, precision=precision, autotune=autotune)

        def batched():
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            _, infos, st = S.solve_batch(A, TOL, psi)
            e[1].record(stream)
            torch.cuda.synchronize(dev)
            assert st == spfd.SPFD_OK, spfd.spfd_last_error()
            return e[0].elapsed_time(e[1]), infos

        def sequential():
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            infos = []
            e[0].record(stream)
            for j in range(nrhs):
                _, info, st = S.solve(A[j], TOL, psi[j])
                assert st == spfd.SPFD_OK, spfd.spfd_last_error()
                infos.append(info)
            e[1].record(stream)
            torch.cuda.synchronize(dev)
            return e[0].elapsed_time(e[1]), infos

        out = {}
        # the first batched call grows the buffers and runs the autotuner
        t0 = time.perf_counter()
        batched()
        out["first_batched_call_ms"] = round((time.perf_counter() - t0) * 1e3, 1)
        todo = (("batched", batched), ("sequential", sequential)) if sequential_too \
            else (("batched", batched),)
        for name, fn in todo:
            for _ in range(W):
                fn()
            rec = [fn() for _ in range(K)]
            ms = statistics.mean(r[0] for r in rec)
            infos = rec[-1][1]
            it = [i["iters"] for i in infos]
            out[name] = {"ms": round(ms, 3), "solves_per_s": round(nrhs / (ms * 1e-3), 2),
                         "iters_mean": round(statistics.mean(it), 2), "iters_max": max(it),
                         "launches": int(sum(i["launches"] for i in infos)) if name == "sequential"
                         else int(infos[0]["launches"]),
                         "max_rel_res_true": max(i["rel_res_true"] for i in infos)}
        out["context_bytes_device"] = S.info()["bytes_device"]
        if sequential_too:
            out["speedup_batched_vs_sequential"] = round(
                out["sequential"]["ms"] / out["batched"]["ms"], 3)
        rep = S.autotune_report()
        if rep:
            out["autotune"] = {
                "decisions": len(rep),
                "orders_chosen": [sum(r["order"] == k for r in rep) for k in range(3)],
                "tuned_launch_ms": {f"{r['family']}_l{r['level']}":
                                    [round(r["ms_order0"], 3), round(r["ms_order1"], 3),
                                     round(r["ms_order2"], 3), r["order"]]
                                    for r in rep},
                "note": "per family and level: [ms per launch in order 0 (right-hand sides one "
                        "after the other), in order 1 (all right-hand sides of a brick side by "
                        "side), in order 2 (tiles of 4 right-hand sides per block, operator "
                        "entries read once per tile; -1 where the family has none), order "
                        "kept]; orders_chosen counts the decisions per order"}
        S.close()
        return out

    fp64 = run(spfd.SPFD_FP64)
    mixed = run(spfd.SPFD_MIXED)
    fp64["batched_fixed_order0_ms"] = run(spfd.SPFD_FP64, 0, False)["batched"]["ms"]
    mixed["batched_fixed_order0_ms"] = run(spfd.SPFD_MIXED, 0, False)["batched"]["ms"]
    del A, psi
    return {"workload": f"{nrhs} loop sources (R=0.3 m, I=1000 A) at seeded positions x,y in "
                        "+-0.5 m, z in -0.6..-0.3 m, random orientations, on the "
                        "256x160x896 body, h=2 mm",
            "nrhs": nrhs, "tol": TOL, "steps": K, "warmup": W,
            "fp64": fp64, "mixed": mixed,
            "mixed_batched_vs_fp64_batched": round(fp64["batched"]["ms"] / mixed["batched"]["ms"], 3)}


def cpu_baseline(ph, a, iters=30, record=None):
    """The oracle (CPU, FP64, as it stands) on a bounded sample of the same
    workload: assembly + right-hand side, `iters` Jacobi-PCG iterations, and
    |E|; the solve is extrapolated to the oracle's own iteration count for
    1e-8 on this workload (tests/golden/body_2mm_oracle.json)."""
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    sys_ = oracle.assemble(ph.sigma, ph.h)
    b = oracle.project(sys_, oracle.rhs(sys_, a))
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    x, info = oracle.pcg(sys_, b, tol=1e-300, maxit=iters)
    t_it = (time.perf_counter() - t0) / max(info["iters"], 1)
    psi = sys_.scatter(oracle.project(sys_, x))
    t0 = time.perf_counter()
    oracle.efield(ph.sigma, a, psi, ph.h, OMEGA)
    t_e = time.perf_counter() - t0
    n_it, src = None, None
    try:
        with open(GOLDEN) as f:
            g = json.load(f)
        n_it = int(g["tol_1e-08"]["iters"])
        src = "tests/golden/body_2mm_oracle.json"
    except Exception:
        pass
    if n_it is None:
        return {"value": None, "unit": "s", "cores": oracle.num_threads(), "kind": "oracle",
                "sample": f"assembly + {info['iters']} Jacobi-PCG iterations ({t_it:.4f} s/iter); "
                          "iteration count to 1e-8 unavailable"}
    total = t_setup + n_it * t_it + t_e
    cores = oracle.num_threads()
    # the same iterations on one core (the solve is where the oracle's time goes)
    one = None
    if cores > 1:
        oracle.set_num_threads(1)
        try:
            t0 = time.perf_counter()
            _, info1 = oracle.pcg(sys_, b, tol=1e-300, maxit=5)
            t1 = (time.perf_counter() - t0) / max(info1["iters"], 1)
        finally:
            oracle.set_num_threads(cores)
        one = {"s_per_iter": round(t1, 4), "solve_s": round(n_it * t1, 2),
               "speedup_of_cores": round(t1 / t_it, 2),
               "sample": f"{info1['iters']} Jacobi-PCG iterations on one thread, extrapolated "
                         f"to the {n_it} iterations to 1e-8"}
    out = {"value": round(total, 3), "unit": "s", "cores": cores, "kind": "oracle",
           "sample": (f"full-size workload: assembly+rhs {t_setup:.2f} s, {info['iters']} Jacobi-PCG "
                      f"iterations timed ({t_it:.4f} s/iter) and extrapolated to the oracle's "
                      f"{n_it} iterations to 1e-8 ({src}), |E| {t_e:.2f} s")}
    if one:
        out["single_core"] = one
    return out


def run_reference(args):
    """The reference arm: the CPU FP64 oracle as it stands, on the host's
    cores, over whole steps of the same workload (assembly and right-hand
    side, Jacobi-PCG to 1e-8, |E|).  After one short warm-up (assembly and 30
    iterations) it times full steps until K are done or the next one would
    pass the time budget (at least one); "steps" is the number of full steps
    timed."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    ph, a = _inputs()
    cores = oracle.num_threads()
    for _ in range(min(args.warmup, 1)):
        sys_ = oracle.assemble(ph.sigma, ph.h)
        oracle.pcg(sys_, oracle.project(sys_, oracle.rhs(sys_, a)), tol=1e-300, maxit=30)
    times, iters = [], []
    t_start = time.perf_counter()
    while len(times) < max(1, args.steps):
        t0 = time.perf_counter()
        psi, info, _ = oracle.solve(ph.sigma, ph.h, a, tol=TOL)
        oracle.efield(ph.sigma, a, psi, ph.h, OMEGA)
        times.append(time.perf_counter() - t0)
        iters.append(info["iters"])
        assert info["converged"]
        if time.perf_counter() - t_start + times[-1] > args.reference_budget_s:
            break
    v = round(statistics.mean(times), 3)
    sample = (f"{len(times)} full step(s) of the workload timed on {cores} host threads: "
              f"assembly + right-hand side, Jacobi-PCG to {TOL:g} ({iters[-1]} iterations), |E|")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": len(times),
            "warmup": args.warmup, "ms_per_step": round(v * 1000, 1),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": DATA, "config": _config(1),
            "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "timing": "host wall clock around each full step"}
    print(json.dumps(line), flush=True)


def run_ncu_step(args):
    """One step (build + solve + |E|) of the full-size workload, nothing else:
    the target of the ncu launch lists and captures summarised in profiles/."""
    import torch

    import paper_2010_12879_gb300 as spfd

    if args.ncu_small:
        # the same body and source at 4 mm: 128 x 80 x 448 voxels, ~1.2M
        # unknowns, stencil arrays still larger than L2
        from spfd_inputs import body_phantom, loop_potential
        ph = body_phantom(128, 80, 448, h=4e-3)
        a = loop_potential(ph.dims, ph.h, ph.origin)
    else:
        ph, a = _inputs()
    sig = torch.from_numpy(ph.sigma).cuda()
    ad = torch.from_numpy(a).cuda()
    prec = spfd.SPFD_FP64 if args.ncu_step == "fp64" else spfd.SPFD_MIXED
    with spfd.Solver(sig, ph.h, precision=prec) as S:
        psi, info, st = S.solve(ad, TOL)
        E = S.efield(ad, psi, OMEGA)
        torch.cuda.synchronize()
        assert st == spfd.SPFD_OK and info["converged"], spfd.spfd_last_error()
    print(json.dumps({"ncu_step": args.ncu_step, "iters": info["iters"],
                      "outer_iters": info["outer_iters"],
                      "rel_res_true": info["rel_res_true"],
                      "launches": info["launches"]}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-iters", type=int, default=30)
    ap.add_argument("--reference-budget-s", type=float, default=150.0,
                    help="--impl reference: stop timing full steps once the next one would "
                         "pass this many seconds")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-percentile", action="store_true")
    ap.add_argument("--no-group", action="store_true")
    ap.add_argument("--no-1mm", action="store_true")
    ap.add_argument("--no-tree-cotree", action="store_true")
    ap.add_argument("--no-chebyshev", action="store_true")
    ap.add_argument("--batch-rhs", type=int, default=64,
                    help="source fields of the batched-solve sub-object")
    ap.add_argument("--ncu-step", choices=["fp64", "mixed"], default=None,
                    help="run one untimed step only (profiling target)")
    ap.add_argument("--ncu-small", action="store_true",
                    help="with --ncu-step: the 4 mm body (128x80x448) instead")
    args = ap.parse_args()
    if args.ncu_step:
        run_ncu_step(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
