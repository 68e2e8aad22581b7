"""Benchmark: tetrahedral elements assembled per second on GB300.

Workload (default): the 100^3-hex unit cube split into 6,000,000 Kuhn tets
(1,030,301 nodes, nnz 15,210,901), interior nodes jittered by +-15% h, node
numbering a seeded random permutation; rho = 1, mu = 1e-3, dt = 1e-2;
velocity = seeded sum of sinusoids.  One step = one full assembly of A
(CSR), G (3 CSR value arrays) and rhs through the C ABI, inputs resident in
HBM, outputs overwritten.  Mixed precision (float gathers and element
arithmetic, compensated accumulation stored as double) is the headline; the
plain FP64 mode is timed beside it.

Prints ONE JSON line (rank 0).  Under torchrun each rank assembles its own
replica of the workload (no data-path collective) and value is the total
over ranks.  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import meshgen  # noqa: E402

WORKLOADS = {
    "batch64": "64 jittered Kuhn cubes, N ~ U{10..60} hexes a side (seeded), one persistent batched launch "
               "captured with the velocity update in a CUDA graph and replayed every step",
    "adjoint50": "Kuhn cube 50^3 hexes, 750,000 tets, jitter 15% h: vector-Jacobian product of R = A(u)u - b",
    "step100": "Kuhn cube 100^3 hexes, 6,000,000 tets, jitter 15% h, random numbering, seed 1: one time step with "
               "cached geometry, A = A_static + C(u) and rhs (A_static and G assembled once, outside the timing)",
    "cube100": "Kuhn cube 100^3 hexes, 6,000,000 tets, 1,030,301 nodes, jitter 15% h, random numbering, seed 1",
    "stab100": "stabilised velocity block (3x3 block per CSR entry: Galerkin part, SUPG product, transposed-"
               "gradient viscous coupling, grad-div term; Codina's tau1, tau2) of the 100^3 cube: 6,000,000 tets, "
               "jitter 15% h, random numbering, seed 1",
    "cube8": "Kuhn cube 8^3 hexes, 3,072 tets, 729 nodes, natural numbering, seed 0",
    "cube70": "Kuhn cube 70^3 hexes, 2,058,000 tets, 357,911 nodes, jitter 15% h, random numbering, seed 1 "
              "(profiling case: the 100^3 recipe with outputs still above L2)",
    "cube200_rcm": "Kuhn cube 200^3 hexes, 48,000,000 tets, 8,120,601 nodes, jitter 15% h, RCM numbering, 5% noise",
    "cube200_random": "Kuhn cube 200^3 hexes, 48,000,000 tets, 8,120,601 nodes, jitter 15% h, random numbering, 5% noise",
}
PREC_BYTES = {"fp64": (8, 8, 8), "mixed64": (8, 4, 8), "mixed32": (8, 4, 4)}  # coord, velocity, output


def algorithmic_bytes(E, n, nnz, precision):
    """Compulsory HBM bytes of one assembly: connectivity 16 B/tet, coordinates,
    velocities, CSR pattern (row_ptr + col_idx), A + 3 G value arrays, 3 rhs."""
    sx, su, so = PREC_BYTES[precision]
    return 16 * E + n * (3 * sx + 3 * su) + 4 * (n + 1) + 4 * nnz + so * 4 * nnz + so * 3 * n


def stab_bytes(E, n, nnz, precision):
    """Compulsory HBM bytes of one stabilised-block assembly: connectivity 16 B/tet,
    coordinates, velocities, CSR pattern, Auu (9 values per entry) + 3 G value
    arrays, 3 rhs."""
    sx, su, so = PREC_BYTES[precision]
    return 16 * E + n * (3 * sx + 3 * su) + 4 * (n + 1) + 4 * nnz + so * 12 * nnz + so * 3 * n


def stab_times(mesh, u, precs, steps, warmup, flush, stream, rows=None, sampler=None):
    """Per precision: ms per nsi_assemble_stabilized call and of its main kernel
    (L2 flushed before every step), elements/s, the HBM roofline of the kernel
    and the largest row-scaled error of sampled rows against the oracle."""
    import torch

    import oracle
    import paper_2111_05651_gb300 as nsi

    E, n = mesh.n_elems, mesh.n_nodes
    peak, _ = hbm_peak()
    res = {}
    for prec in precs:
        asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=prec)
        vt = torch.float64 if prec == "fp64" else torch.float32
        ut = torch.as_tensor(u.T.copy()).to("cuda", vt).contiguous()
        out = (torch.empty(9, asm.nnz, dtype=asm.out_dtype, device="cuda"),
               torch.empty(3, asm.nnz, dtype=asm.out_dtype, device="cuda"),
               torch.empty(3, n, dtype=asm.out_dtype, device="cuda"))
        fn = lambda: asm.assemble_stabilized(ut, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT, out=out)  # noqa
        if sampler is not None and prec == precs[0]:
            sampler.mark("t0")
        ms, kms = time_steps(asm, fn, steps if prec != "fp64" else max(3, min(steps, 5)), warmup, flush, stream)
        if sampler is not None and prec == precs[0]:
            sampler.mark("t1")
        km = statistics.mean(kms)
        nb = stab_bytes(E, n, asm.nnz, prec)
        info = asm.info()
        rec = {"ms": statistics.mean(ms), "kernel_ms": km, "elements_per_s": E / (statistics.mean(ms) * 1e-3),
               "algorithmic_bytes": nb, "achieved_gbs": nb / (km * 1e-3) / 1e9,
               "roofline_frac": nb / (km * 1e-3) / 1e9 / peak, "kernel": "stab_star_kernel",
               # pack, the row kernel, then the per-row kernel for long rows and
               # (mixed modes) for the rows of badly shaped elements, if any
               "launches_per_step": 2 + (info.long_rows > 0) + (prec != "fp64" and info.exact_rows > 0)}
        if rows is not None:
            uo = u if prec == "fp64" else u.astype(np.float32).astype(np.float64)
            ref = oracle.assemble_stabilized_rows(mesh.coord, mesh.lnods, uo, rows, None, meshgen.RHO, meshgen.MU,
                                                  meshgen.DT)
            rp = asm.pattern()[0].cpu().numpy()
            Auu, G, rh = (t.double().cpu().numpy() for t in out)
            err = 0.0
            for r, (cols, blk, g, orh) in zip(rows, ref):
                s_, e_ = rp[r], rp[r + 1]
                for c in range(9):
                    err = max(err, np.abs(Auu[c, s_:e_] - blk[c]).max() / np.abs(blk[c]).max())
                for d in range(3):
                    err = max(err, np.abs(G[d, s_:e_] - g[d]).max() / np.abs(g[d]).max())
                err = max(err, np.abs(rh[:, r] - orh).max() / np.abs(rh).max())
            rec["max_rel_err"] = float(err)
        res[prec] = rec
        asm.close()
        del out
    return res


def run_stab(args, world, rank, local):
    import torch

    import paper_2111_05651_gb300 as nsi

    torch.cuda.set_device(local)
    nsi.load_library()
    mesh, u = meshgen.config_mesh("cube100")
    E, n = mesh.n_elems, mesh.n_nodes
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rows = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(9).integers(0, n, 24)]))
    precs = [args.precision] + ([p for p in ("mixed32", "mixed64", "fp64") if p != args.precision]
                                if not args.quick else [])
    sampler = ClockSampler(local)
    sampler.start()
    barrier(world)
    res = stab_times(mesh, u, precs, args.steps, args.warmup, lambda: flush_buf.fill_(1),
                     torch.cuda.current_stream(), rows, sampler)
    barrier(world)
    clocks = sampler.stop()
    m = res[args.precision]
    ms = allreduce_max(m["ms"], world)
    if "fp64" in res:  # FP64 mode against the FP64 pipe
        res["fp64"]["fp64_roofline"] = fp64_roofline(E, res["fp64"]["kernel_ms"], STAB_FP64_FLOPS_PER_TET)
    if rank == 0:
        peak, src = hbm_peak()
        print(json.dumps({"metric": "tet elements assembled/s (stabilised velocity block)",
                          "value": world * E / (ms * 1e-3), "unit": "elements/s", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None,
                          "dtype": {"fp64": "f64", "mixed64": "f32", "mixed32": "f32"}[args.precision],
                          "data": "synthetic",
                          "config": {"workload": WORKLOADS["stab100"], "precision": args.precision,
                                     "elements": E, "nodes": n,
                                     "l2": "flushed (256 MiB write) before every timed step"},
                          "roofline": {"bound": "hbm", "achieved": m["achieved_gbs"], "peak": peak, "unit": "GB/s",
                                       "frac": m["achieved_gbs"] / peak,
                                       "traffic": read_traffic("stab_star_kernel", "cube100", args.precision),
                                       "kernel": "stab_star_kernel", "algorithmic_bytes": m["algorithmic_bytes"],
                                       "kernel_ms": m["kernel_ms"], "peak_source": src},
                          "clocks": clocks, "gpu_launches": args.steps * m["launches_per_step"],
                          "max_rel_err": m.get("max_rel_err"), "modes": res}), flush=True)


def csrc_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2111_05651_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def read_traffic(kernel, workload, precision):
    """ncu DRAM bytes per launch, committed under profiles/, if taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f)
        key = f"{kernel}|{workload}|{precision}"
        r = rec.get(key)
        if r and r.get("csrc_hash") == csrc_hash():
            return r["dram_bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        pass
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while it runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, period_ms=20):
        self.index, self.period, self.lines, self.proc, self.t0, self.t1 = index, period_ms, [], None, None, None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 f"-lms", str(self.period)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)  # let the first samples arrive

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "note": "nvidia-smi unavailable"}
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        inside = [l for (t, l) in self.lines if self.t0 is not None and self.t0 <= t <= self.t1 + 0.05]
        note = None
        if len(inside) < 2:
            # the timed region is shorter than the sampling period: take the samples next to it
            near = sorted(self.lines, key=lambda x: abs(x[0] - (self.t0 or x[0])))[:4]
            inside = [l for _, l in near]
            note = "timed region shorter than the sampling period; nearest samples used"
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in inside:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
                power.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
               "samples": len(sm), "power_w_max": max(power) if power else None}
        if note:
            out["note"] = note
        return out


def dist_setup(cpu_only=False):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        gpu = torch.cuda.is_available() and not cpu_only
        if gpu:
            torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl" if gpu else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    on_gpu = torch.cuda.is_available() and dist.get_backend() == "nccl"
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if on_gpu else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------- CPU oracle ---
def cpu_oracle_rate(mesh, u, n_elems, repeats=3, threads=1):
    """Elements/s of the FP64 oracle on the first n_elems tets: the serial
    assembly on one host thread, or the multi-threaded one (bitwise the same
    result) on `threads` threads (0: every host core)."""
    import oracle

    ln = mesh.lnods[:n_elems]
    csr = oracle.pattern(mesh.n_nodes, ln)
    times = []
    for _ in range(repeats):
        t = time.perf_counter()
        if threads == 1:
            oracle.assemble(mesh.coord, ln, u, None, meshgen.RHO, meshgen.MU, meshgen.DT, csr=csr)
        else:
            oracle.assemble_threads(mesh.coord, ln, u, None, meshgen.RHO, meshgen.MU, meshgen.DT, csr=csr,
                                    threads=threads)
        times.append(time.perf_counter() - t)
    return n_elems / statistics.median(times), statistics.median(times)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle

    mesh, u = meshgen.config_mesh(args.workload if args.workload in meshgen.CONFIGS else "cube100")
    n_s = min(args.ref_sample, mesh.n_elems)
    ln = mesh.lnods[:n_s]
    csr = oracle.pattern(mesh.n_nodes, ln)
    cores = host_cores()

    def one():
        oracle.assemble_threads(mesh.coord, ln, u, None, meshgen.RHO, meshgen.MU, meshgen.DT, csr=csr,
                                threads=cores)

    for _ in range(args.warmup):
        one()
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        one()
        times.append(time.perf_counter() - t)
    ms = 1e3 * statistics.mean(times)
    value = n_s / (ms * 1e-3)
    sample = (f"first {n_s} of {mesh.n_elems} tets of the workload per step (all nodes), FP64, "
              f"{cores} host threads (OpenMP; bitwise the serial oracle's result)")
    line = {
        "impl": "reference", "metric": "tet elements assembled/s", "value": value, "unit": "elements/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "precision": "fp64 oracle", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "elements/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- GPU ---
def time_steps(asm, fn, steps, warmup, flush, stream):
    """Per-step device time of the whole call and of its main assembly kernel
    (ms), with an L2 flush before every step (outside both timings)."""
    import torch

    for _ in range(warmup):
        flush()
        fn()
    torch.cuda.synchronize()
    mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    step_ev = [(mk(), mk()) for _ in range(steps)]
    kern_ev = [(mk(), mk()) for _ in range(steps)]
    for k in range(steps):
        asm.set_timing_events(*kern_ev[k])
    torch.cuda.synchronize()
    for k in range(steps):
        flush()
        asm.set_timing_events(*kern_ev[k])
        step_ev[k][0].record(stream)
        fn()
        step_ev[k][1].record(stream)
    torch.cuda.synchronize()
    asm.set_timing_events(None, None)
    return ([a.elapsed_time(b) for a, b in step_ev], [a.elapsed_time(b) for a, b in kern_ev])


def max_sampled_error(asm, mesh, u_gpu_f64, out, rows):
    """Row-scaled error of sampled rows against the oracle (full-size check)."""
    import oracle

    A, G, rhs = (t.double().cpu().numpy() for t in out)
    rp, ci = (t.cpu().numpy() for t in asm.pattern())
    ref = oracle.assemble_rows(mesh.coord, mesh.lnods, u_gpu_f64, rows, None, meshgen.RHO, meshgen.MU, meshgen.DT)
    worst = 0.0
    for r, (cols, a, g, rh) in zip(rows, ref):
        s, e = rp[r], rp[r + 1]
        assert np.array_equal(ci[s:e], cols)
        worst = max(worst, np.abs(A[s:e] - a).max() / np.abs(a).max())
        for d in range(3):
            worst = max(worst, np.abs(G[d, s:e] - g[d]).max() / np.abs(g[d]).max())
    return float(worst)


def run_gpu(args, world, rank, local):
    import torch

    import paper_2111_05651_gb300 as nsi

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nsi.load_library()
    mesh, u = meshgen.config_mesh(args.workload)
    E, n = mesh.n_elems, mesh.n_nodes
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def flush():
        flush_buf.fill_(1)

    results = {}
    main_prec = args.precision
    precs = [main_prec] + ([p for p in ("fp64", "mixed32", "mixed64") if p != main_prec] if not args.quick else [])
    for prec in precs:
        asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=prec, scatter=args.scatter)
        if args.fan:
            nsi.nsi_set_launch(asm.handle, nsi.NSI_SCATTER_GATHER, -1)
        if args.atomic_agg:
            nsi.nsi_set_launch(asm.handle, nsi.NSI_SCATTER_ATOMIC, 1)
        vt = torch.float64 if prec == "fp64" else torch.float32
        ut = torch.as_tensor(u.T.copy()).to(dev, vt).contiguous()
        out = asm.empty_outputs()
        fn = lambda: asm.assemble(ut, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT, out=out)  # noqa: E731
        steps = args.steps if prec == main_prec else max(3, min(args.steps, 10))
        sampler = ClockSampler(local) if prec == main_prec else None
        if sampler:
            sampler.start()
        for _ in range(args.warmup):
            flush()
            fn()
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        if sampler:
            sampler.mark("t0")
        ms, kms = time_steps(asm, fn, steps, 0, flush, stream)
        torch.cuda.synchronize()
        if sampler:
            sampler.mark("t1")
        barrier(world)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        mean_ms = statistics.mean(ms)
        mode = {0: "auto", 1: "color", 2: "atomic", 3: "gather"}[asm.scatter]
        rec = {"ms": mean_ms, "ms_min": min(ms), "ms_median": statistics.median(ms), "steps": steps,
               "kernel_ms": statistics.mean(kms), "elements_per_s": E / (mean_ms * 1e-3), "clocks": clocks,
               "nnz": asm.nnz, "mode": mode, "persistent": bool(asm.info().persistent),
               "launches_per_step": {"gather": 2, "atomic": 1, "color": asm.n_colors}[mode]}
        if not args.quick or prec == main_prec:
            rows = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(7).integers(0, n, 48)]))
            uo = u if prec == "fp64" else u.astype(np.float32).astype(np.float64)
            rec["max_rel_err"] = max_sampled_error(asm, mesh, uo, out, rows)
            if prec != "fp64":
                rec["max_rel_err_vs_f64_inputs"] = max_sampled_error(asm, mesh, u, out, rows)
        if prec == main_prec and not args.no_e2e:
            # end to end through the C ABI with host buffers
            uh = torch.as_tensor(u.T.copy()).to(vt).pin_memory()
            Ah = torch.empty(asm.nnz, dtype=asm.out_dtype).pin_memory()
            Gh = torch.empty(3, asm.nnz, dtype=asm.out_dtype).pin_memory()
            rh = torch.empty(3, n, dtype=asm.out_dtype).pin_memory()
            asm.assemble_host(uh, Ah, Gh, rh, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT)
            k_e2e = max(3, min(args.steps, 10))
            barrier(world)
            t = time.perf_counter()
            for _ in range(k_e2e):
                asm.assemble_host(uh, Ah, Gh, rh, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT)
            e2e_s = (time.perf_counter() - t) / k_e2e
            e2e_s = allreduce_max(e2e_s, world)
            osz = Ah.element_size()
            rec["e2e"] = {"value": world * E / e2e_s, "unit": "elements/s",
                          "h2d_bytes_per_step": int(uh.numel() * uh.element_size()),
                          "d2h_bytes_per_step": int(osz * (4 * asm.nnz + 3 * n)), "ms_per_step": 1e3 * e2e_s}
        results[prec] = rec
        asm.close()
        del out

    main = results[main_prec]
    ms_max = allreduce_max(main["ms"], world)
    value = world * E / (ms_max * 1e-3)
    gather_name = "fan_kernel" if args.fan else ("gather_persistent_kernel" if main["persistent"] else "gather_kernel")
    kernel = {"gather": gather_name, "atomic": "elem_kernel",
              "color": "elem_kernel"}[main["mode"]]
    bytes_alg = algorithmic_bytes(E, n, main["nnz"], main_prec)
    peak, peak_src = hbm_peak()
    achieved = bytes_alg / (main["kernel_ms"] * 1e-3) / 1e9
    line = {
        "metric": "tet elements assembled/s", "value": value, "unit": "elements/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed64": "f32", "mixed32": "f32"}[main_prec],
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "precision": main_prec, "scatter": main["mode"],
                   "output_dtype": {"fp64": "f64", "mixed64": "f64", "mixed32": "f32"}[main_prec],
                   "elements": E, "nodes": n, "nnz": main["nnz"],
                   "l2": "flushed (256 MiB write) before every timed step; working set > L2",
                   "replicas": "each rank assembles its own copy of the workload" if world > 1 else None},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": read_traffic(kernel, args.workload, main_prec), "kernel": kernel,
                     "algorithmic_bytes": bytes_alg, "kernel_ms": main["kernel_ms"],
                     "peak_source": peak_src},
        "clocks": main["clocks"],
        "gpu_launches": args.steps * main["launches_per_step"],
        "max_rel_err": main.get("max_rel_err"),
        "max_rel_err_vs_f64_inputs": main.get("max_rel_err_vs_f64_inputs"),
        "modes": {p: {k: r[k] for k in ("ms", "kernel_ms", "elements_per_s", "max_rel_err", "mode") if k in r}
                  for p, r in results.items()},
    }
    if "fp64" in results and main_prec != "fp64":
        line["speedup_vs_fp64"] = results["fp64"]["ms"] / main["ms"]
    if "e2e" in main:
        line["e2e"] = main["e2e"]
    if "fp64" in results:
        line["fp64_roofline"] = fp64_roofline(E, results["fp64"]["kernel_ms"])
    if rank == 0 and not args.no_cpu_baseline:
        n_s = min(args.cpu_sample, E)
        cores = host_cores()
        rate, med = cpu_oracle_rate(mesh, u, n_s, threads=cores)
        line["cpu_baseline"] = {"value": rate, "unit": "elements/s", "cores": cores, "kind": "oracle",
                                "sample": f"first {n_s} tets of the workload (all nodes), FP64, median of 3 runs of "
                                          f"{med:.2f} s each, {cores} host threads (OpenMP element pass, then a row "
                                          f"pass in element order: bitwise the serial oracle's result)"}
        rate1, med1 = cpu_oracle_rate(mesh, u, n_s, threads=1)
        line["cpu_baseline_1core"] = {"value": rate1, "unit": "elements/s", "cores": 1, "kind": "oracle",
                                      "sample": f"the same sample, serial oracle, median of 3 runs of {med1:.2f} s"}
    if world == 1 and not args.no_extras and args.workload == "cube100":
        line["more_workloads"] = more_workloads(args, (mesh, u))
    if rank == 0:
        print(json.dumps(line), flush=True)


# FP64 floating-point operations per tet of the FP64 row gather, counted from
# its double-precision arithmetic (an FMA is 2): each element is evaluated from
# each of its 4 rows, 96 per evaluation (two cofactor cross products 18, det 5,
# c_i 9, 1/det by Newton-Raphson 9, the viscous factor 1, the convection-plus-
# viscous vector w 18, the pressure-gradient vector 3, three w . c_x 15 with
# their orientation 4, the row's accumulators 12, the determinant sum 2), plus
# the per-row diagonal sums and edge vectors (about 20 per tet at 5.8 tets per
# node).  The method's own count (each element once) is about 300.
FP64_FLOPS_PER_TET = 4 * 96 + 20


def fp64_peak():
    """(TFLOP/s, source): cuBLAS DGEMM (4096^3, best of 3) measured in this run."""
    import torch

    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return 2.0 * n ** 3 / best / 1e12, "cuBLAS DGEMM 4096^3 measured in this run (best of 3)"


# FP64 floating-point operations per tet of the stabilised row kernel in FP64
# mode, counted from its double-precision arithmetic (an FMA is 2; cbrt and
# sqrt counted as 1 each, their own operations not counted): each element is
# evaluated once per row, 166 per evaluation (three cofactor cross products
# 27, det 5, c_i 6, 1/det by Newton-Raphson 8, the viscous factor 1, the
# velocity sum 9 and its norm 5, tau's lengths 3, the SUPG factor 12, the
# grad-div factor 3, five SUPG dot products with their scaling 30, the
# Galerkin-plus-SUPG vector 42, three dot products 15), and added into each of
# its 12 directed entries, 47 per addition (the nine coupling components 42,
# G 3, A + S and det 2).  The rows' diagonal blocks and the write-out are not
# counted.
STAB_FP64_FLOPS_PER_TET = 4 * 166 + 12 * 47


def fp64_roofline(E, kernel_ms, flops_per_tet=FP64_FLOPS_PER_TET):
    """FP64 mode's bound: the double-precision pipe.  achieved = the kernel's
    FP64 operations (flops_per_tet x tets) / its time, against DGEMM."""
    peak, src = fp64_peak()
    achieved = flops_per_tet * E / (kernel_ms * 1e-3) / 1e12
    return {"bound": "fp64", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "flops_per_tet": flops_per_tet, "kernel_ms": kernel_ms, "peak_source": src}


def more_workloads(args, mesh100=None):
    """Compact records of the largest single-GPU workload (the 200^3 cube in RCM
    numbering, 48 M tets, mixed32 and mixed64 row gather), of the stabilised
    velocity block on the 100^3 cube (mixed64), of the batching workload (64
    meshes, graph replay) and of the adjoint case (50^3 cube, VJP in FP64 and
    mixed64): ms per step, elements/s and, for the assemblies, the HBM
    roofline fraction of the main kernel."""
    import torch

    import paper_2111_05651_gb300 as nsi

    out = {}
    t_start = time.perf_counter()
    mesh, u = meshgen.config_mesh("cube200_rcm")
    E, n = mesh.n_elems, mesh.n_nodes
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    peak, _ = hbm_peak()
    rec = {"workload": WORKLOADS["cube200_rcm"], "elements": E, "steps": 10, "modes": {}}
    for prec in ("mixed32", "mixed64"):
        asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=prec)
        ut = torch.as_tensor(u.T.copy()).cuda().float().contiguous()
        o = asm.empty_outputs()
        fn = lambda: asm.assemble(ut, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT, out=o)  # noqa: E731
        ms, kms = time_steps(asm, fn, 10, 3, lambda: flush_buf.fill_(1), stream)
        km = statistics.mean(kms)
        b = algorithmic_bytes(E, n, asm.nnz, prec)
        rec["modes"][prec] = {"ms": statistics.mean(ms), "kernel_ms": km,
                              "elements_per_s": E / (statistics.mean(ms) * 1e-3),
                              "roofline_frac": b / (km * 1e-3) / 1e9 / peak}
        asm.close()
        del o
    out["cube200_rcm"] = rec
    del mesh, u
    torch.cuda.empty_cache()
    if mesh100 is not None:
        res = stab_times(mesh100[0], mesh100[1], ("mixed64",), 20, 3, lambda: flush_buf.fill_(1), stream)
        out["stab100"] = {"workload": WORKLOADS["stab100"], "elements": mesh100[0].n_elems, "steps": 20,
                          "modes": res}
    out["batch64"] = batch_record(steps=100, warmup=5, precision="mixed64", autotune=True)
    E, res = adjoint_times(50, 5)
    out["adjoint50"] = {"workload": WORKLOADS["adjoint50"], "elements": E, "steps": 50,
                        "l2": "flushed (256 MiB write) before every call", "modes": res}
    out["seconds"] = time.perf_counter() - t_start
    return out


def shard_meshes(sizes, world):
    """Independent meshes split over ranks, largest first to the least-loaded
    rank (element counts balanced); every mesh goes to exactly one rank."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    loads = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += sizes[i]
    return [sorted(p) for p in parts]


def batch_time(precision, autotune, warmup, steps, world=1, rank=0):
    """64 meshes per step: velocity update + batched assembly replayed from one
    CUDA graph.  With N ranks the meshes are split over the ranks (no
    collective).  Returns (ms per step, max over ranks; elements of the whole
    batch; autotuned launch shapes; meshes on this rank)."""
    import torch

    import paper_2111_05651_gb300 as nsi

    all_meshes = meshgen.batch_meshes()
    mine = shard_meshes([m.n_elems for m, _ in all_meshes], world)[rank]
    meshes = [all_meshes[i] for i in mine]
    asms = [nsi.Assembler(m.coord, m.lnods, precision=precision) for m, _ in meshes]
    vt = torch.float64 if precision == "fp64" else torch.float32
    base = [torch.as_tensor(u.T.copy()).cuda().to(vt) for _, u in meshes]
    cache = os.path.join(ROOT, "paper_2111_05651_gb300", "_build", "autotune_cache.json") if autotune else None
    tuned = {}
    if autotune:
        for a, b in zip(asms, base):
            r = a.autotune(b, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT, cache=cache)
            tuned[r] = tuned.get(r, 0) + 1
    cur = [b.clone() for b in base]
    outs = [a.empty_outputs() for a in asms]
    step = torch.zeros(1, device="cuda", dtype=vt)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        nsi.assemble_batched(asms, cur, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT, outs=outs)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step.add_(1.0)
        for c, b in zip(cur, base):  # u(t) = u0 cos(2 pi 0.01 t): the in-graph velocity update
            c.copy_(b * torch.cos(0.06283185307179587 * step))
        nsi.assemble_batched(asms, cur, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT, outs=outs)
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize()
    E = sum(m.n_elems for m, _ in all_meshes)  # the whole batch, over all ranks
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    ms = allreduce_max(e0.elapsed_time(e1) / steps, world)
    del graph
    for a in asms:
        a.close()
    return ms, E, tuned, len(meshes)


def batch_record(steps, warmup, precision, autotune):
    """The batching workload as a compact record (one GPU)."""
    ms, E, tuned, _ = batch_time(precision, autotune, warmup, steps)
    return {"workload": WORKLOADS["batch64"], "elements": E, "precision": precision, "steps": steps,
            "ms": ms, "elements_per_s": E / (ms * 1e-3),
            "autotuned": {f"{k[0]}/{k[1]}": v for k, v in tuned.items()} or None}


def run_batch(args, world, rank, local):
    import torch

    import paper_2111_05651_gb300 as nsi

    torch.cuda.set_device(local)
    nsi.load_library()
    prec = args.precision
    ms, E, tuned, n_mine = batch_time(prec, args.autotune, args.warmup, args.steps, world, rank)
    if rank == 0:
        print(json.dumps({
            "metric": "tet elements assembled/s", "value": E / (ms * 1e-3), "unit": "elements/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS["batch64"], "meshes": 64, "elements": E,
                       "meshes_on_rank0": n_mine,
                       "precision": prec, "launches_per_step": "1 batched + 1 batched pack + velocity update",
                       "autotuned": {f"{k[0]}/{k[1]}": v for k, v in tuned.items()} or None,
                       "l2": "working set (outputs of all meshes) > L2; no flush between replays"},
        }), flush=True)


def adjoint_times(steps, warmup):
    """The 50^3 adjoint case: per VJP call (FP64 and mixed64), device time by
    CUDA events around each call with the L2 flushed before it; the median
    and mean ms, and elements/s at the median."""
    import torch

    import paper_2111_05651_gb300 as nsi

    mesh, u = meshgen.config_mesh("cube50")
    w = meshgen.gaussian_weights(mesh.n_nodes, np.random.default_rng(40))
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res = {}
    for prec in ("fp64", "mixed64"):
        asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=prec)
        vt = torch.float64 if prec == "fp64" else torch.float32
        ut = torch.as_tensor(u.T.copy()).cuda().to(vt)
        wt = torch.as_tensor(w.T.copy()).cuda().to(vt)
        for _ in range(warmup):
            flush_buf.fill_(1)
            asm.vjp(ut, wt, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush_buf.fill_(1)
            e0.record()
            asm.vjp(ut, wt, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT)
            e1.record()
        torch.cuda.synchronize()
        ms = [e0.elapsed_time(e1) for e0, e1 in ev]
        med = statistics.median(ms)
        res[prec] = {"ms": med, "ms_mean": statistics.mean(ms), "elements_per_s": mesh.n_elems / (med * 1e-3)}
        asm.close()
    return mesh.n_elems, res


def run_adjoint(args, world, rank, local):
    import torch

    import paper_2111_05651_gb300 as nsi

    torch.cuda.set_device(local)
    nsi.load_library()
    E, res = adjoint_times(args.steps, args.warmup)
    if rank == 0:
        print(json.dumps({"metric": "tet elements differentiated/s (VJP of the assembled residual)",
                          "value": res["mixed64"]["elements_per_s"], "unit": "elements/s", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["mixed64"]["ms"],
                          "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                          "config": {"workload": WORKLOADS["adjoint50"], "elements": E},
                          "modes": res}), flush=True)


def hbm_peak():
    """(GB/s, source) of the HBM roofline: the measured copy bandwidth, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured hbm_gbs (copy, burst)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s, one earlier GB300 measurement)"


def step_bytes(E, n, nnz, precision):
    """Compulsory HBM bytes of one cached-geometry step: connectivity, node data,
    row_ptr + col_idx, A_static read and A written, rhs written."""
    sx, su, so = PREC_BYTES[precision]
    return 16 * E + n * (3 * sx + 3 * su) + 4 * (n + 1) + 4 * nnz + 2 * so * nnz + 3 * so * n


def run_step(args, world, rank, local):
    import torch

    import oracle
    import paper_2111_05651_gb300 as nsi

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nsi.load_library()
    mesh, u = meshgen.config_mesh("cube100")
    E, n = mesh.n_elems, mesh.n_nodes
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    rows = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(9).integers(0, n, 24)]))
    res = {}
    for prec in ("mixed64", "mixed32", "fp64"):
        asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=prec)
        vt = torch.float64 if prec == "fp64" else torch.float32
        ut = torch.as_tensor(u.T.copy()).to(dev, vt).contiguous()
        A_static, _ = asm.static_part(rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT)
        out = (torch.empty_like(A_static), torch.empty(3, n, dtype=asm.out_dtype, device=dev))
        fn = lambda: asm.assemble_convective(ut, A_static, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT,  # noqa
                                             out=out)
        steps = args.steps if prec == "mixed64" else max(3, min(args.steps, 20))
        sampler = ClockSampler(local) if prec == "mixed64" else None
        if sampler:
            sampler.start()
            sampler.mark("t0")
        t_step, t_kern = time_steps(asm, fn, steps, args.warmup, lambda: flush_buf.fill_(1), stream)
        if sampler:
            sampler.mark("t1")
        clocks = sampler.stop() if sampler else None
        ms, kms = float(np.mean(t_step)), float(np.mean(t_kern))
        # sampled rows of A and rhs against the oracle's full assembly
        u_in = u if prec == "fp64" else u.astype(np.float32).astype(np.float64)
        ref = oracle.assemble_rows(mesh.coord, mesh.lnods, u_in, rows, None, meshgen.RHO, meshgen.MU, meshgen.DT)
        rp = asm.pattern()[0].cpu().numpy()
        Ah, rh = out[0].double().cpu().numpy(), out[1].double().cpu().numpy()
        err = 0.0
        for r, (cols, a, g, orh) in zip(rows, ref):
            err = max(err, np.abs(Ah[rp[r]:rp[r + 1]] - a).max() / np.abs(a).max(),
                      np.abs(rh[:, r] - orh).max() / np.abs(rh).max())
        nb = step_bytes(E, n, asm.nnz, prec)
        res[prec] = {"ms": ms, "kernel_ms": kms, "elements_per_s": E / (ms * 1e-3), "max_rel_err": float(err),
                     "algorithmic_bytes": nb, "achieved_gbs": nb / (kms * 1e-3) / 1e9}
        if clocks is not None:
            res[prec]["clocks"] = clocks
        asm.close()
    ms = allreduce_max(res["mixed64"]["ms"], world)
    if rank == 0:
        peak, src = hbm_peak()
        m = res["mixed64"]
        print(json.dumps({"metric": "tet elements stepped/s (cached-geometry convective step)",
                          "value": world * E / (ms * 1e-3), "unit": "elements/s", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                          "scaling": "weak", "dtype": "f32", "data": "synthetic",
                          "config": {"workload": WORKLOADS["step100"], "precision": "mixed64",
                                     "l2": "flushed (256 MiB write) before every timed step"},
                          "roofline": {"bound": "hbm", "achieved": m["achieved_gbs"], "peak": peak, "unit": "GB/s",
                                       "frac": m["achieved_gbs"] / peak,
                                       "traffic": read_traffic("step_kernel", "cube100", "mixed64"), "kernel": "step_kernel",
                                       "algorithmic_bytes": m["algorithmic_bytes"], "kernel_ms": m["kernel_ms"],
                                       "peak_source": src},
                          "clocks": m.pop("clocks", None), "gpu_launches": args.steps * 2,  # pack + step kernel
                          "max_rel_err": m["max_rel_err"], "modes": res}), flush=True)


def run_profile(args):
    """Untimed assemblies for an external profiler: per precision, 3 calls."""
    import torch

    import paper_2111_05651_gb300 as nsi

    nsi.load_library()
    mesh, u = meshgen.config_mesh(args.workload)
    for prec in args.profile_run.split(","):
        asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=prec, scatter=args.scatter)
        if args.fan:
            nsi.nsi_set_launch(asm.handle, nsi.NSI_SCATTER_GATHER, -1)
        if args.atomic_agg:
            nsi.nsi_set_launch(asm.handle, nsi.NSI_SCATTER_ATOMIC, 1)
        vt = torch.float64 if prec == "fp64" else torch.float32
        ut = torch.as_tensor(u.T.copy()).cuda().to(vt)
        if args.profile_stab:  # the stabilised velocity block: 3 calls
            out = (torch.empty(9, asm.nnz, dtype=asm.out_dtype, device="cuda"),
                   torch.empty(3, asm.nnz, dtype=asm.out_dtype, device="cuda"),
                   torch.empty(3, mesh.n_nodes, dtype=asm.out_dtype, device="cuda"))
            for _ in range(3):
                asm.assemble_stabilized(ut, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT, out=out)
        elif args.profile_step:  # the cached-geometry time step: A_static once, then 3 steps
            A_static, _ = asm.static_part(rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT)
            step_out = (torch.empty_like(A_static), torch.empty(3, mesh.n_nodes, dtype=asm.out_dtype, device="cuda"))
            for _ in range(3):
                asm.assemble_convective(ut, A_static, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT, out=step_out)
        else:
            out = asm.empty_outputs()
            for _ in range(3):
                asm.assemble(ut, rho=meshgen.RHO, mu=meshgen.MU, dt=meshgen.DT, out=out)
        torch.cuda.synchronize()
        asm.close()
    print("profile run done", args.workload, args.profile_run)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cube100", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="mixed64", choices=["fp64", "mixed64", "mixed32"])
    ap.add_argument("--scatter", default="auto", choices=["auto", "gather", "color", "atomic"])
    ap.add_argument("--cpu-sample", type=int, default=3_000_000)
    ap.add_argument("--ref-sample", type=int, default=3_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the 200^3 and batch64 records of the default run")
    ap.add_argument("--quick", action="store_true", help="time only the main precision")
    ap.add_argument("--autotune", action="store_true", help="batch64: autotune launch shapes (cached)")
    ap.add_argument("--fan", action="store_true", help="row gather through the edge-fan kernel")
    ap.add_argument("--atomic-agg", action="store_true", help="atomic scatter with warp-aggregated atomics")
    ap.add_argument("--profile-step", action="store_true", help="--profile-run times the cached-geometry step")
    ap.add_argument("--profile-stab", action="store_true", help="--profile-run runs the stabilised velocity block")
    ap.add_argument("--profile-run", default=None, metavar="PRECS",
                    help="no timing: 3 assembly calls per listed precision (for ncu)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.profile_run:
        run_profile(args)
        return
    world, rank, local = dist_setup(cpu_only=args.impl == "reference")
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        elif args.workload == "batch64":
            run_batch(args, world, rank, local)
        elif args.workload == "adjoint50":
            run_adjoint(args, world, rank, local)
        elif args.workload == "step100":
            run_step(args, world, rank, local)
        elif args.workload == "stab100":
            run_stab(args, world, rank, local)
        else:
            run_gpu(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
