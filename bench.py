"""Benchmark of the HPS direct solver on one GB300 (or N, as independent replicas).

A step is one pass of the whole hot path: the build (leaf operators, then
every merge level up to the root) followed by one solve (upward and downward
sweeps) for one right-hand side, on the 16 x 16-leaf workload (p = 16, q = 14,
kappa = eta = 80, periodic medium, eight Gaussian point sources, t = 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` = DOF built and solved per second over
the K timed steps (inputs resident in HBM, L2 flushed between steps), plus
separate build DOF/s, solve RHS/s and p50/p99 single-RHS solve latency.  The
`reference` implementation is the plain CPU oracle on the host cores.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1812_07167_gb300 import replicas  # noqa: E402
from paper_1812_07167_gb300 import workloads as W  # noqa: E402

METRIC = "HPS build DOF/s and solve RHS/s at stated rel. error; p50/p99 solve latency"
M, P_ORDER, KAPPA = 16, 16, 80.0
# FP64 peak from unit counts: 2 FP64 FMA a clock per SM (4 flop) on this part,
# times the SM count the device reports and its maximum SM clock (152 SMs at
# 2.07 GHz: the 1.25 TFLOP/s nominal of the part)
FP64_FLOP_PER_CLK_PER_SM = 4


def workload():
    return W.point_sources(m=M, p=P_ORDER, kappa=KAPPA)


def config_dict(nrhs=1):
    """The workload of a step, the same for both arms (the GPU path and the
    reference arm, the oracle on the host cores); how each arm computes it is
    in implementation_dict."""
    wl = workload()
    return {
        "workload": "helmholtz_impedance_point_sources",
        "leaves": f"{M}x{M}", "p": P_ORDER, "q": P_ORDER - 2, "kappa": KAPPA, "eta": KAPPA,
        "c": "1+0.3 sin(4 pi x) cos(6 pi y)", "s": "8 Gaussian sources, width 0.01, seed 1", "t": 0,
        "dof": M * M * (P_ORDER * P_ORDER - 4), "tensor_nodes": M * M * P_ORDER * P_ORDER,
        "nrhs_per_step": nrhs, "precision": "complex128",
        "l2": "GPU arm: L2 flushed between timed steps (256 MiB write); host-core arm: not applicable",
        "domain": list(wl.domain),
    }


def implementation_dict(gpu=True):
    """How an arm computes the step: the GPU path's leaf form and products,
    or the reference arm's program."""
    if not gpu:
        return {"program": "the oracle (oracle/hps_oracle.c): Algorithm 1 and 2 in plain C99 complex128, "
                           "dense LU per leaf, OpenMP over the boxes of a level"}
    return {
        "leaf_form": ("LU factors P D B = L U (leaf kernel), two triangular sweeps a solve" if LEAF_FORM == 0
                      else "B^-1: complex64 Gauss-Jordan inverse refined to complex128 by two steps of "
                           "E = I - B X (Ozaki product on tcgen05) and X += X0 E; one product a solve"),
        "products": ("FP64 pipes; merge products of 2^26+ complex multiply-adds by the Ozaki scheme "
                     "on the bf16 tensor cores (tcgen05; 9 slices of 6 bits, exact FP32 slice sums, "
                     "complex128 totals)"),
    }


class ClockSampler:
    """nvidia-smi samples (every 50 ms) while the timed region runs: the
    sampler is started, its first sample awaited (at most 5 s) and dropped,
    so that every kept sample falls inside the region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.skip = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
            self.skip = len(self.lines)
        except OSError:
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
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.skip:]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_oracle_step(c, s, t, threads):
    import oracle as O

    wl = workload()
    pr = O.Problem(wl.m, wl.p, wl.kappa, wl.eta)
    t0 = time.perf_counter()
    T = O.Tree(pr, c, nthreads=threads)
    u = T.solve(s[None], t[None], nthreads=threads)[0]
    dt = time.perf_counter() - t0
    R = T.root_R()
    cond = T.cond_W()
    T.close()
    return dt, u, R, cond


def reference_arm(args, rank, world):
    """The plain CPU oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    import oracle as O

    wl = workload()
    pr = O.Problem(wl.m, wl.p, wl.kappa, wl.eta)
    lxy, bxy = O.nodes(pr)
    c, s, t = wl.sample(lxy, bxy)
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        run_oracle_step(c, s, t, threads)
    times = [run_oracle_step(c, s, t, threads)[0] for _ in range(args.steps)]
    dof = pr.leaves * pr.n
    total = sum(times)
    value = dof * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(), "implementation": implementation_dict(gpu=False),
        "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": threads, "kind": "oracle",
                         "sample": "full 16x16-leaf build + 1-RHS solve per step"},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


LEAF_FORM = 1  # hps.HPS_LEAF_INVERSE (the default); --leaf-form lu sets HPS_LEAF_LU


def _problem(*args, **kw):
    """hps.Problem with the leaf form chosen on the command line."""
    from paper_1812_07167_gb300 import hps

    return hps.Problem(*args, leaf_form=LEAF_FORM, **kw)


def ours(args, rank, world, local_rank):
    import torch

    from paper_1812_07167_gb300 import hps

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
    st = torch.cuda.current_stream()
    wl = workload()
    pr = _problem(wl.m, wl.p, wl.kappa, wl.eta)
    lxy, bxy = hps.hps_nodes(pr)
    c, s, t = wl.sample(lxy, bxy)
    cd = torch.from_numpy(c).to(dev)
    sd = torch.from_numpy(np.ascontiguousarray(s[None])).to(dev)
    td = torch.from_numpy(np.ascontiguousarray(t[None])).to(dev)
    ud = torch.empty((1, pr.leaves, pr.n), dtype=torch.complex128, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def step():
        h = hps.hps_build(pr, cd, st)
        hps.hps_solve(h, sd, td, ud, 1, st)
        return h

    # measured kernel choices for this problem's shapes (kept for the process)
    t_tune = time.perf_counter()
    tuned_shapes = hps.hps_tune([pr], st)
    tune_s = time.perf_counter() - t_tune

    for _ in range(max(args.warmup, 3)):
        h = step()
        torch.cuda.synchronize()
        code, lev, box = hps.hps_status(h, st)
        if code != hps.HPS_OK:
            raise RuntimeError(f"build reported {hps.hps_strerror(code)} at level {lev} box {box}")
        h.free()
    h0 = step()
    torch.cuda.synchronize()
    info = h0.info()
    h0.free()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    leaf_ms = []
    prod_times = []  # per timed step: (ms, bf16 flops) of each tensor-core product kernel
    handles = []
    with ClockSampler(local_rank) as clk:  # started (first sample seen) before the barrier
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(st)
            h = step()
            ev[k][1].record(st)
            handles.append(h)
            if len(handles) > 1:  # free the previous step's operators outside the timed pair
                torch.cuda.synchronize()
                leaf_ms.append(hps.hps_build_times(handles[0])[0])
                prod_times.append(hps.hps_build_product_times(handles[0]))
                handles.pop(0).free()
        torch.cuda.synchronize()
        t_wall1 = time.perf_counter()
    if dist:
        dist.barrier()  # every rank's timed region has ended
    for hh in handles:
        leaf_ms.append(hps.hps_build_times(hh)[0])
        prod_times.append(hps.hps_build_product_times(hh))
        hh.free()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dof = pr.leaves * pr.n
    all_units, total_ms = replicas.aggregate(dof * args.steps, sum(step_ms), dev)
    value = all_units / (total_ms / 1e3)

    # ---- separate build / solve figures (device-resident inputs) ----
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    build_ms = []
    for _ in range(10):
        flush.zero_()
        e0.record(st)
        h = hps.hps_build(pr, cd, st)
        e1.record(st)
        torch.cuda.synchronize()
        build_ms.append(e0.elapsed_time(e1))
        h.free()
    h = hps.hps_build(pr, cd, st)
    # latency as a caller sees it: the call plus a wait on the stream; device
    # time from events around the call on the same stream
    lat, lat_dev = [], []
    for k in range(220):
        st.synchronize()
        t0 = time.perf_counter()
        e0.record(st)
        hps.hps_solve(h, sd, td, ud, 1, st)
        e1.record(st)
        st.synchronize()
        t1 = time.perf_counter()
        if k >= 20:
            lat.append((t1 - t0) * 1e3)
            lat_dev.append(e0.elapsed_time(e1))
    nb = 64
    S = sd.repeat(nb, 1, 1).contiguous()
    T = td.repeat(nb, 1).contiguous()
    U = torch.empty((nb, pr.leaves, pr.n), dtype=torch.complex128, device=dev)
    for _ in range(2):
        hps.hps_solve(h, S, T, U, nb, st)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(5):
        hps.hps_solve(h, S, T, U, nb, st)
    e1.record(st)
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1) / 5
    u_gpu = ud.cpu().numpy()[0]
    R_gpu = np.zeros((pr.nbdry, pr.nbdry), complex)
    hps.hps_root_R(h, R_gpu, st)
    h.free()

    # ---- end to end through the C ABI with pinned host buffers ----
    cp = torch.from_numpy(c).pin_memory()
    sp = torch.from_numpy(np.ascontiguousarray(s[None])).pin_memory()
    tp = torch.from_numpy(np.ascontiguousarray(t[None])).pin_memory()
    upin = torch.empty((1, pr.leaves, pr.n), dtype=torch.complex128).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hh = hps.hps_build(pr, cp.numpy(), st)
        hps.hps_solve(hh, sp.numpy(), tp.numpy(), upin.numpy(), 1, st)  # returns once u is on the host
        t1 = time.perf_counter()
        hh.free()
        if k >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_value = replicas.throughput(dof * len(e2e_ms), sum(e2e_ms), dev)

    # ---- mixed-precision path on the same problem (complex64 leaves and lower
    # merges, complex128 top levels and refinement) ----
    pm = _problem(wl.m, wl.p, wl.kappa, wl.eta, precision=hps.HPS_MIXED)
    mb = []
    for _ in range(4):
        flush.zero_()
        e0.record(st)
        hm = hps.hps_build(pm, cd, st)
        e1.record(st)
        torch.cuda.synchronize()
        mb.append(e0.elapsed_time(e1))
        hm.free()
    hm = hps.hps_build(pm, cd, st)
    um = torch.empty_like(ud)
    mlat = []
    for k in range(60):
        st.synchronize()
        t0 = time.perf_counter()
        hps.hps_solve(hm, sd, td, um, 1, st)
        st.synchronize()
        if k >= 10:
            mlat.append((time.perf_counter() - t0) * 1e3)
    Um = torch.empty_like(U)
    hps.hps_solve(hm, S, T, Um, nb, st)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(5):
        hps.hps_solve(hm, S, T, Um, nb, st)
    e1.record(st)
    torch.cuda.synchronize()
    mbatch_ms = e0.elapsed_time(e1) / 5
    u_mixed = um.cpu().numpy()[0]
    R_mixed = np.zeros_like(R_gpu)
    hps.hps_root_R(hm, R_mixed, st)
    minfo = hm.info()
    hm.free()

    # ---- the other leaf form on the same problem (LU factors vs B^-1): its
    # build, 1-RHS latency and 64-RHS rate, and its u against this run's ----
    po = hps.Problem(wl.m, wl.p, wl.kappa, wl.eta, leaf_form=1 - LEAF_FORM)
    ob = []
    for _ in range(4):
        flush.zero_()
        e0.record(st)
        ho = hps.hps_build(po, cd, st)
        e1.record(st)
        torch.cuda.synchronize()
        ob.append(e0.elapsed_time(e1))
        ho.free()
    ho = hps.hps_build(po, cd, st)
    uo = torch.empty_like(ud)
    olat = []
    for k in range(60):
        st.synchronize()
        t0 = time.perf_counter()
        hps.hps_solve(ho, sd, td, uo, 1, st)
        st.synchronize()
        if k >= 10:
            olat.append((time.perf_counter() - t0) * 1e3)
    Uo = torch.empty_like(U)
    hps.hps_solve(ho, S, T, Uo, nb, st)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(5):
        hps.hps_solve(ho, S, T, Uo, nb, st)
    e1.record(st)
    torch.cuda.synchronize()
    obatch_ms = e0.elapsed_time(e1) / 5
    u_other = uo.cpu().numpy()[0]
    ho.free()
    other = {
        "leaf_form": "B^-1 (Gauss-Jordan)" if LEAF_FORM == 0 else "LU factors",
        "build_ms_median": statistics.median(ob), "build_dof_per_s": dof / (statistics.median(ob) / 1e3),
        "solve_rhs_per_s": nb / (obatch_ms / 1e3), "solve_nrhs_batch": nb,
        "solve_latency_ms_p50": float(np.percentile(olat, 50)),
        "rel_diff_u_vs_this_form": float(np.abs(u_other - u_gpu).max() / np.abs(u_gpu).max()),
    }

    batch_res = None if args.no_batching else batching(dev, st, flush)
    # the 64 x 64-leaf, kappa = 300 workload (FP64 and mixed; the oracle's
    # comparison is added on rank 0 below)
    c3 = c3_data = None
    if world == 1 and not args.no_config3:
        c3, c3_data = precision_run(dev, st, flush)
    fp64_measured = hps.hps_fp64_rate(st)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count

    if rank != 0:
        return
    lu = LEAF_FORM == 0
    leaf_avg = statistics.mean(leaf_ms)
    clocks = clk.summary()
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    fp64_nominal = n_sm * FP64_FLOP_PER_CLK_PER_SM * max_mhz * 1e6 / 1e12
    if lu:
        # the dominant kernel is the LU leaf kernel, bound by the FP64 pipes:
        # LU of [B; G] and the G-row solve (one complex multiply-add = 8 flop)
        leaf_kernel = "lu_leaf_kernel"
        leaf_flops = pr.leaves * 8 * (pr.n ** 3 // 3 + pr.nb * pr.n ** 2)
        achieved = leaf_flops / (leaf_avg / 1e3) / 1e12
        traffic = stored_traffic(leaf_kernel)
        roofline = {"kernel": leaf_kernel, "bound": "alu", "achieved": achieved, "flops_per_launch": leaf_flops,
                    "peak": fp64_nominal, "unit": "TFLOP/s", "frac": achieved / fp64_nominal,
                    "traffic": traffic, "leaf_ms": leaf_avg,
                    "peak_source": f"FP64 unit count x max SM clock ({n_sm} SMs x "
                                   f"{FP64_FLOP_PER_CLK_PER_SM} flop/clk x {max_mhz:.0f} MHz)",
                    "peak_measured": fp64_measured, "frac_of_measured": achieved / fp64_measured,
                    "peak_measured_source": "hps_fp64_rate: independent FMA chains on every SM, CUDA events"}
    else:
        # the dominant kernel is the tensor-core product (oz_tc_kernel); its
        # largest launches are the leaf step's residuals E = I - B X (n x n x n
        # over the leaves, the first products of a build), timed by the events
        # the build records around each product kernel
        steps_refine = 2
        lead = [(ms[:steps_refine], fl[:steps_refine]) for ms, fl in prod_times]
        r_ms = sum(float(m.sum()) for m, _ in lead)
        r_fl = sum(float(f.sum()) for _, f in lead)
        n_launch = sum(len(m) for m, _ in lead)
        achieved = r_fl / (r_ms / 1e3) / 1e12
        all_ms = sum(float(m.sum()) for m, _ in prod_times)
        all_fl = sum(float(f.sum()) for _, f in prod_times)
        bf16_peak, peak_src = bf16_peak_sustained()
        roofline = {"kernel": "oz_tc_kernel", "bound": "tensor", "achieved": achieved,
                    "flops_per_launch": r_fl / max(n_launch, 1), "unit": "TFLOP/s", "peak": bf16_peak,
                    "frac": achieved / bf16_peak, "traffic": stored_traffic("oz_tc_kernel"),
                    "launch_ms": r_ms / max(n_launch, 1), "launches_timed": n_launch,
                    "what": f"the leaf residual products E = I - B X ({pr.n} x {pr.n} x {pr.n} over {pr.leaves} "
                            "leaves, bf16 slice flops = 45 pairs x 4 real products x 2 M N K), CUDA events "
                            "around each product kernel on the build's stream",
                    "peak_source": peak_src,
                    "all_tensor_core_products": {"launches_per_step": len(prod_times[0][0]) if prod_times else 0,
                                                 "achieved": all_fl / (all_ms / 1e3) / 1e12,
                                                 "frac": all_fl / (all_ms / 1e3) / 1e12 / bf16_peak},
                    "leaf_phase_ms": leaf_avg}
    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded point sources; no dataset)", "config": config_dict(),
        "implementation": implementation_dict(),
        "build_dof_per_s": dof / (statistics.median(build_ms) / 1e3),
        "build_ms_median": statistics.median(build_ms),
        "solve_rhs_per_s": nb / (batch_ms / 1e3), "solve_nrhs_batch": nb,
        "solve_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                             "device_p50": float(np.percentile(lat_dev, 50)),
                             "device_p99": float(np.percentile(lat_dev, 99)),
                             "nrhs": 1, "samples": len(lat),
                             "what": "wall clock of hps_solve + stream sync, device-resident s, t, u"},
        "operator_bytes": info.operator_bytes, "build_flops": info.build_flops,
        "tuning": {"shapes": tuned_shapes, "seconds": tune_s,
                   "what": "hps_tune: measured tile / tensor-core choice per merge product shape and "
                           "cluster / panel regime per interface-inverse shape, before the timed steps"},
        "roofline": roofline,
        "fp64_peak": {"nominal": fp64_nominal, "measured": fp64_measured,
                      "nominal_source": f"{n_sm} SMs x {FP64_FLOP_PER_CLK_PER_SM} flop/clk x {max_mhz:.0f} MHz",
                      "measured_source": "hps_fp64_rate"},
        "e2e": {"value": e2e_value, "unit": "DOF/s",
                "h2d_bytes_per_step": int(c.nbytes + s.nbytes + t.nbytes),
                "d2h_bytes_per_step": int(u_gpu.nbytes)},
        "gpu_launches": args.steps * (info.build_launches + info.solve_launches),
        "clocks": clocks,
        "wall_s_timed_region": t_wall1 - t_wall0,
        "mixed": {
            "what": "complex64 leaves and lower merges, complex128 top 4 levels, 2 complex128 refinement steps",
            "build_dof_per_s": dof / (statistics.median(mb) / 1e3), "build_ms_median": statistics.median(mb),
            "solve_rhs_per_s": nb / (mbatch_ms / 1e3),
            "solve_latency_ms": {"p50": float(np.percentile(mlat, 50)), "p99": float(np.percentile(mlat, 99)),
                                 "nrhs": 1, "samples": len(mlat)},
            "rel_err_u_vs_fp64_gpu": float(np.abs(u_mixed - u_gpu).max() / np.abs(u_gpu).max()),
            "rel_err_root_R_vs_fp64_gpu": float(np.linalg.norm(R_mixed - R_gpu) / np.linalg.norm(R_gpu)),
            "operator_bytes": minfo.operator_bytes,
        },
        "other_leaf_form": other,
        "batching": batch_res,
    }
    if world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        dt, u_ora, R_ora, cond_ora = run_oracle_step(c, s, t, threads)
        line["cpu_baseline"] = {"value": dof / dt, "unit": "DOF/s", "cores": threads, "kind": "oracle",
                                "sample": "one full 16x16-leaf build + 1-RHS solve"}
        # the same oracle on one thread, for the scale of its OpenMP speedup
        dt1 = run_oracle_step(c, s, t, 1)[0]
        line["cpu_baseline_single_thread"] = {"value": dof / dt1, "unit": "DOF/s", "cores": 1, "kind": "oracle",
                                              "sample": "one full 16x16-leaf build + 1-RHS solve"}
        line["rel_err_vs_oracle"] = {
            "u": float(np.abs(u_gpu - u_ora).max() / np.abs(u_ora).max()),
            "root_R": float(np.linalg.norm(R_gpu - R_ora) / np.linalg.norm(R_ora)),
            # conditioning that bounds the agreement of two correct FP64 builds
            "cond1_W_per_level_from_root": [float(f"{v:.3g}") for v in cond_ora],
        }
        line["mixed"]["rel_err_u_vs_oracle"] = float(np.abs(u_mixed - u_ora).max() / np.abs(u_ora).max())
        line["mixed"]["rel_err_root_R_vs_oracle"] = float(np.linalg.norm(R_mixed - R_ora) / np.linalg.norm(R_ora))
        if c3 is not None:
            precision_oracle(c3, c3_data)
    if c3 is not None:
        line["config3_64x64"] = c3
    print(json.dumps(line), flush=True)


def batching(dev, st, flush, reps=2):
    """Ragged batch of 32 independent problems (m in {8, 16, 32}, p = 16,
    kappa = eta in [20, 200], random media, seeds 100..131): the batch built by
    one hps_build_batch call against the same problems built one hps_build
    after another, FP64 and mixed; device time with CUDA events."""
    import torch

    from paper_1812_07167_gb300 import hps

    spec = W.ragged_batch()
    out = {"problems": len(spec), "m": [m for m, _, _ in spec], "p": P_ORDER,
           "dof": sum(m * m * (P_ORDER * P_ORDER - 4) for m, _, _ in spec)}
    cs = []
    for m, kap, cfun in spec:
        lxy, _ = hps.hps_nodes(_problem(m, P_ORDER, kap, kap))
        nb = 4 * (P_ORDER - 2)
        cs.append(torch.from_numpy(cfun(lxy[:, nb:, 0], lxy[:, nb:, 1])).to(dev))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    us = {}
    for name, prec in (("fp64", hps.HPS_FP64), ("mixed", hps.HPS_MIXED)):
        probs = [_problem(m, P_ORDER, kap, kap, precision=prec) for m, kap, _ in spec]
        res = {}
        # measured kernel choices for the batch's shapes and for each size alone
        res["tuned_shapes"] = hps.hps_tune(probs, st) + sum(
            hps.hps_tune([_problem(m, P_ORDER, 50.0, 50.0, precision=prec)], st) for m in sorted({m for m, _, _ in spec}))
        for mode in ("batched", "separate"):
            ms = []
            for rep in range(reps + 1):
                flush.zero_()
                e0.record(st)
                if mode == "batched":
                    hs = hps.hps_build_batch(probs, cs, st)
                else:
                    hs = [hps.hps_build(pr, c, st) for pr, c in zip(probs, cs)]
                e1.record(st)
                torch.cuda.synchronize()
                if rep:
                    ms.append(e0.elapsed_time(e1))
                if rep == reps:
                    k = max(range(len(spec)), key=lambda i: spec[i][0])
                    _, s1, t1 = W.random_data(spec[k][0], P_ORDER, spec[k][1], spec[k][1], seed=9)
                    u = torch.empty((1, spec[k][0] ** 2, P_ORDER * P_ORDER - 4), dtype=torch.complex128, device=dev)
                    hps.hps_solve(hs[k], torch.from_numpy(s1[None]).to(dev), torch.from_numpy(t1[None]).to(dev), u, 1, st)
                    us[(name, mode)] = u.cpu().numpy()
                    res[f"{mode}_launches"] = (hs[0].info().build_launches if mode == "batched"
                                               else sum(h.info().build_launches for h in hs))
                for h in hs:
                    h.free()
            res[f"{mode}_ms"] = statistics.median(ms)
            res[f"{mode}_dof_per_s"] = out["dof"] / (statistics.median(ms) / 1e3)
        # new coefficients for the same batch: the build replayed as one CUDA graph
        hs = hps.hps_build_batch(probs, cs, st)
        hps.hps_rebuild(hs, cs, st)  # captures the graph
        torch.cuda.synchronize()
        ms = []
        for rep in range(reps):
            flush.zero_()
            e0.record(st)
            hps.hps_rebuild(hs, cs, st)
            e1.record(st)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        res["rebuild_graph_ms"] = statistics.median(ms)
        for h in hs:
            h.free()
        res["speedup"] = res["separate_ms"] / res["batched_ms"]
        a, b = us[(name, "batched")], us[(name, "separate")]
        res["rel_diff_u_batched_vs_separate"] = float(np.abs(a - b).max() / np.abs(b).max())
        out[name] = res
    a, b = us[("mixed", "batched")], us[("fp64", "batched")]
    out["mixed"]["rel_err_u_vs_fp64"] = float(np.abs(a - b).max() / np.abs(b).max())
    return out


def precision_run(dev, st, flush):
    """64 x 64 leaves (1,032,192 unknowns), p = 16, kappa = eta = 300, random
    medium (seed 2) with 8 Gaussian sources, t = 0: the complex128 path
    against the mixed path (complex64 leaves and lower merges, complex128 top
    4 levels, complex128 refinement), on the GPU.  Returns the JSON part and
    what precision_oracle needs to add the oracle's figures."""
    import torch

    from paper_1812_07167_gb300 import hps

    m, p, kappa = 64, P_ORDER, 300.0
    wl = W.random_medium_sources(m, p, kappa)
    pr = _problem(m, p, kappa, kappa)
    lxy, bxy = hps.hps_nodes(pr)
    c, s, t = wl.sample(lxy, bxy)
    cd = torch.from_numpy(c).to(dev)
    sd = torch.from_numpy(np.ascontiguousarray(s[None])).to(dev)
    td = torch.from_numpy(np.ascontiguousarray(t[None])).to(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dof = pr.leaves * pr.n
    out = {"config": {"workload": "helmholtz_random_medium_sources", "leaves": f"{m}x{m}", "p": p, "q": p - 2,
                      "kappa": kappa, "eta": kappa, "c": "random medium, 32 Fourier modes, seed 2",
                      "s": "8 Gaussian sources, width 0.01", "t": 0, "dof": dof}}
    res = {}
    for name, prec in (("fp64", hps.HPS_FP64), ("mixed", hps.HPS_MIXED)):
        q = _problem(m, p, kappa, kappa, precision=prec)
        tuned = hps.hps_tune([q], st)
        bms = []
        for rep in range(4):
            flush.zero_()
            e0.record(st)
            h = hps.hps_build(q, cd, st)
            e1.record(st)
            torch.cuda.synchronize()
            if rep:
                bms.append(e0.elapsed_time(e1))
            if rep < 3:
                h.free()
        code = hps.hps_status(h, st)[0]
        u = torch.empty((1, pr.leaves, pr.n), dtype=torch.complex128, device=dev)
        sms = []
        for rep in range(6):
            flush.zero_()
            e0.record(st)
            hps.hps_solve(h, sd, td, u, 1, st)
            e1.record(st)
            torch.cuda.synchronize()
            if rep:
                sms.append(e0.elapsed_time(e1))
        R = np.zeros((pr.nbdry, pr.nbdry), complex)
        hps.hps_root_R(h, R, st)
        info = h.info()
        res[name] = {"u": u.cpu().numpy()[0], "R": R}
        out[name] = {"status": hps.hps_strerror(code), "build_ms": statistics.median(bms),
                     "build_dof_per_s": dof / (statistics.median(bms) / 1e3),
                     "solve_ms_1rhs": statistics.median(sms), "solve_rhs_per_s": 1e3 / statistics.median(sms),
                     "operator_bytes": info.operator_bytes, "build_launches": info.build_launches,
                     "tuned_shapes": tuned,
                     "leaf_and_level_ms": [round(float(x), 3) for x in hps.hps_build_times(h)]}
        h.free()
    uf, um = res["fp64"]["u"], res["mixed"]["u"]
    Rf, Rm = res["fp64"]["R"], res["mixed"]["R"]
    out["mixed"]["rel_err_u_vs_fp64_gpu"] = float(np.abs(um - uf).max() / np.abs(uf).max())
    out["mixed"]["rel_err_root_R_vs_fp64_gpu"] = float(np.linalg.norm(Rm - Rf) / np.linalg.norm(Rf))
    return out, (c, s, t, res)


def precision_oracle(out, data):
    """Add to precision_run's result the oracle's full 64 x 64-leaf build +
    solve on the host cores (its time is the CPU baseline) and the errors of
    both GPU paths against it."""
    import oracle as O

    c, s, t, res = data
    m, p, kappa = 64, P_ORDER, 300.0
    dof = m * m * (p * p - 4)
    threads = os.cpu_count() or 1
    opr = O.Problem(m, p, kappa, kappa)
    t0 = time.perf_counter()
    T = O.Tree(opr, c, nthreads=threads)
    uo = T.solve(s[None], t[None], nthreads=threads)[0]
    dt = time.perf_counter() - t0
    Ro = T.root_R()
    cond = T.cond_W()
    T.close()
    out["cpu_baseline"] = {"value": dof / dt, "unit": "DOF/s", "cores": threads, "kind": "oracle",
                           "sample": "one full 64x64-leaf build + 1-RHS solve", "seconds": dt}
    out["cond1_W_per_level_from_root"] = [float(f"{v:.3g}") for v in cond]
    for name in ("fp64", "mixed"):
        out[name]["rel_err_u_vs_oracle"] = float(np.abs(res[name]["u"] - uo).max() / np.abs(uo).max())
        out[name]["rel_err_root_R_vs_oracle"] = float(np.linalg.norm(res[name]["R"] - Ro) / np.linalg.norm(Ro))
    return out


def precision(args, local_rank):
    """The 64 x 64-leaf, kappa = 300 run of precision_run as its own JSON line."""
    import torch

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    st = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    with ClockSampler(local_rank) as clk:
        res, data = precision_run(dev, st, flush)
    out = {"metric": "HPS build DOF/s and solve RHS/s at stated rel. error (64x64 leaves, FP64 vs mixed)",
           "unit": "DOF/s", "higher_is_better": True, "n_gpus": 1, "data": "synthetic"}
    out.update(res)
    out["clocks"] = clk.summary()
    out["value"] = out["mixed"]["build_dof_per_s"]
    if not args.no_cpu_baseline:
        precision_oracle(out, data)
    print(json.dumps(out), flush=True)


def zgemm(args, local_rank):
    """One complex GEMM C = A B (M x K times K x N, batch 1 or the given batch) through
    hps_zgemm: the Ozaki-scheme product on the bf16 tensor cores against the
    FP64-pipe product, device time from CUDA events (median of 5 after 2
    warm-ups), with the relative difference of the two results."""
    import torch

    from paper_1812_07167_gb300 import hps

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    st = torch.cuda.current_stream()
    M, N, K = args.zgemm[:3]
    batch = args.zgemm[3] if len(args.zgemm) > 3 else 1
    g = torch.Generator(device=dev).manual_seed(7)
    A = torch.randn((batch, K, M), dtype=torch.complex128, device=dev, generator=g)
    B = torch.randn((batch, N, K), dtype=torch.complex128, device=dev, generator=g)
    out = {"metric": "complex GEMM rate (FP64-equivalent flops: 8 M N K)", "unit": "TFLOP/s",
           "higher_is_better": True, "n_gpus": 1, "data": "synthetic (normal entries)",
           "config": {"workload": "zgemm", "M": M, "N": N, "K": K, "batch": batch}}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Cs = {}
    for name, emu in (("fp64_pipes", 0), ("tensor_cores", 1)):
        C = torch.empty((batch, N, M), dtype=torch.complex128, device=dev)
        ts = []
        for rep in range(7):
            e0.record(st)
            hps.hps_zgemm(A, B, C, emu, st)
            e1.record(st)
            torch.cuda.synchronize()
            if rep >= 2:
                ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        out[name] = {"ms": ms, "tflops": 8.0 * M * N * K * batch / (ms / 1e3) / 1e12}
        Cs[name] = C
    a, b = Cs["tensor_cores"], Cs["fp64_pipes"]
    out["rel_diff"] = float(((a - b).abs().max() / b.abs().max()).item())
    out["value"] = out["tensor_cores"]["tflops"]
    # bf16 slice products the emulation issues: 45 pairs x 4 real products
    out["tensor_cores"]["bf16_tflops"] = out["tensor_cores"]["tflops"] * 45
    print(json.dumps(out), flush=True)


def scaling(args, local_rank):
    """Build and solve times across leaf counts (4 x 4 ... 128 x 128, p = 16,
    kappa = eta = 80, the point-source workload at each size) for the LU and
    inverse leaf forms in complex128 and the inverse form on the mixed path:
    one JSON line per problem.  Builds: median of 3 (2 at 128 x 128) after the
    problem's kernel choices are measured; solves with device-resident
    vectors, 1 RHS (median of 10) and a wide batch (64 RHS, 16 at 128 x 128)."""
    import torch

    from paper_1812_07167_gb300 import hps

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    st = torch.cuda.current_stream()
    for m in (4, 8, 16, 32, 64, 128):
        wl = W.point_sources(m=m, p=P_ORDER, kappa=KAPPA)
        for form, prec in ((hps.HPS_LEAF_LU, hps.HPS_FP64), (hps.HPS_LEAF_INVERSE, hps.HPS_FP64),
                           (hps.HPS_LEAF_INVERSE, hps.HPS_MIXED)):
            pr = hps.Problem(m, P_ORDER, KAPPA, KAPPA, precision=prec, leaf_form=form)
            lxy, bxy = hps.hps_nodes(pr)
            c, s, t = wl.sample(lxy, bxy)
            cd = torch.from_numpy(c).to(dev)
            hps.hps_tune([pr], st)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            bt = []
            for _ in range(3 if m < 128 else 2):
                e0.record(st)
                h = hps.hps_build(pr, cd, st)
                e1.record(st)
                torch.cuda.synchronize()
                bt.append(e0.elapsed_time(e1))
                h.free()
            h = hps.hps_build(pr, cd, st)
            sd = torch.from_numpy(np.ascontiguousarray(s[None])).to(dev)
            td = torch.from_numpy(np.ascontiguousarray(t[None])).to(dev)
            ud = torch.empty((1, pr.leaves, pr.n), dtype=torch.complex128, device=dev)
            lt = []
            for k in range(12):
                e0.record(st)
                hps.hps_solve(h, sd, td, ud, 1, st)
                e1.record(st)
                torch.cuda.synchronize()
                if k >= 2:
                    lt.append(e0.elapsed_time(e1))
            R = 64 if m <= 64 else 16
            S = sd.repeat(R, 1, 1).contiguous()
            T = td.repeat(R, 1).contiguous()
            U = torch.empty((R, pr.leaves, pr.n), dtype=torch.complex128, device=dev)
            hps.hps_solve(h, S, T, U, R, st)
            torch.cuda.synchronize()
            e0.record(st)
            hps.hps_solve(h, S, T, U, R, st)
            e1.record(st)
            torch.cuda.synchronize()
            wide = e0.elapsed_time(e1)
            info = h.info()
            h.free()
            del S, T, U
            torch.cuda.empty_cache()
            dof = pr.leaves * pr.n
            print(json.dumps({"m": m, "leaf_form": "lu" if form == hps.HPS_LEAF_LU else "inverse",
                              "precision": "fp64" if prec == hps.HPS_FP64 else "mixed",
                              "build_ms": statistics.median(bt), "build_dof_per_s": dof / (statistics.median(bt) / 1e3),
                              "solve_1rhs_ms": statistics.median(lt), "wide_nrhs": R, "wide_ms": wide,
                              "wide_rhs_per_s": R / (wide / 1e3), "operator_bytes": info.operator_bytes}), flush=True)


def polynomial(args, local_rank):
    """Capacity check: an m x m-leaf problem (p = 16, kappa = eta = 40) whose
    exact solution is a polynomial of degree p - 1 in x and y, which the
    discretisation reproduces at every node to rounding.  Builds it twice
    (CUDA events), solves once and reports the largest nodal error against
    the polynomial and the device memory in use.  At m = 256 the host
    sampling of s and t takes a few minutes."""
    import torch

    from paper_1812_07167_gb300 import hps

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    st = torch.cuda.current_stream()
    m = args.polynomial
    wl = W.polynomial_solution(m, P_ORDER, 40.0, 40.0)
    pr = _problem(m, P_ORDER, wl.kappa, wl.eta)
    lxy, bxy = hps.hps_nodes(pr)
    c, s, t = wl.sample(lxy, bxy)
    ue = wl.u_exact(lxy[..., 0], lxy[..., 1])
    info = hps.hps_plan(pr)
    cd = torch.from_numpy(c).to(dev)
    hps.hps_tune([pr], st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bt = []
    for k in range(2):
        e0.record(st)
        h = hps.hps_build(pr, cd, st)
        e1.record(st)
        torch.cuda.synchronize()
        bt.append(e0.elapsed_time(e1))
        code = hps.hps_status(h, st)[0]
        if code != hps.HPS_OK:
            raise RuntimeError(hps.hps_strerror(code))
        phases = hps.hps_build_times(h)
        if k == 0:
            h.free()
    sd = torch.from_numpy(np.ascontiguousarray(s[None])).to(dev)
    td = torch.from_numpy(np.ascontiguousarray(t[None])).to(dev)
    ud = torch.empty((1, pr.leaves, pr.n), dtype=torch.complex128, device=dev)
    for _ in range(3):
        e0.record(st)
        hps.hps_solve(h, sd, td, ud, 1, st)
        e1.record(st)
        torch.cuda.synchronize()
    solve_ms = e0.elapsed_time(e1)
    free, total = torch.cuda.mem_get_info()
    u = ud.cpu().numpy()[0]
    h.free()
    dof = pr.leaves * pr.n
    print(json.dumps({"workload": "polynomial solution", "m": m, "p": P_ORDER, "dof": dof,
                      "leaf_form": "lu" if LEAF_FORM == 0 else "inverse",
                      "build_ms": min(bt), "build_dof_per_s": dof / (min(bt) / 1e3),
                      "build_phases_ms": [float(x) for x in phases], "solve_1rhs_ms": solve_ms,
                      "rel_err_u_vs_polynomial": float(np.abs(u - ue).max() / np.abs(ue).max()),
                      "operator_bytes": info.operator_bytes, "device_bytes_in_use": total - free}), flush=True)


def serving_run(args, local_rank, precision):
    """Config-5 serving workload: a 128 x 128-leaf solver (p = 16, kappa = eta
    = 600, random medium, seed 3) resident in HBM, and a Poisson stream of
    requests: 90% solves of 1..64 right-hand sides (8 seeded Gaussian sources
    each, t = 0), 10% builds of 16 x 16 .. 64 x 64-leaf problems (kappa uniform
    in [20, 200], random medium).  Capacity = requests per second with every
    request queued at once; then the same requests arrive as a Poisson
    process at 50% and 90% of that capacity."""
    import torch

    from paper_1812_07167_gb300 import hps, serve

    dev = torch.device("cuda", local_rank)
    m, p, kappa = args.serve_m, P_ORDER, 600.0
    # the resident solver only solves (wide batches): leaf operators as B^-1,
    # whose product runs on the tensor cores; the build requests take the
    # leaf form given on the command line (B^-1 by default, the faster build)
    pr = hps.Problem(m, p, kappa, kappa, precision=precision,
                     leaf_form=hps.HPS_LEAF_INVERSE if args.serve_resident_form == "inverse" else hps.HPS_LEAF_LU)
    lxy, _ = hps.hps_nodes(pr)
    nb = pr.nb
    xi, yi = lxy[:, nb:, 0], lxy[:, nb:, 1]
    c = W.random_medium(3)(xi, yi)
    st = torch.cuda.current_stream()
    t0 = time.perf_counter()
    h = hps.hps_build(pr, torch.from_numpy(c).to(dev), st)
    code = hps.hps_status(h, st)[0]
    build_s = time.perf_counter() - t0
    if code != hps.HPS_OK:
        raise RuntimeError(f"resident build: {hps.hps_strerror(code)}")
    del c
    pool_n, distinct = 64, 8
    S = torch.empty((pool_n, pr.leaves, pr.ni), dtype=torch.complex128, device=dev)
    for k in range(distinct):
        src, _ = W.gaussian_sources(4000 + k)
        S[k] = torch.from_numpy(src(xi, yi))
    for k in range(distinct, pool_n):
        S[k] = S[k % distinct]
    T = torch.zeros((pool_n, pr.nbdry), dtype=torch.complex128, device=dev)
    sched = W.request_stream(4, args.serve_requests, 1.0)
    builds = {}
    for k, d in enumerate(sched):
        if d["kind"] == "build":
            bp = _problem(d["m"], p, d["kappa"], d["kappa"], precision=precision)
            bx, _ = hps.hps_nodes(bp)
            bc = W.random_medium(d["seed"])(bx[:, nb:, 0], bx[:, nb:, 1])
            builds[k] = (bp, torch.from_numpy(bc).to(dev))
    torch.cuda.synchronize()

    def make(rate):
        out = []
        for k, d in enumerate(W.request_stream(4, args.serve_requests, rate)):
            if d["kind"] == "solve":
                r = d["nrhs"]
                o = (7 * k) % (pool_n - r + 1)
                out.append(serve.Request(k, d["arrival"], "solve", key="main", nrhs=r, s=S[o:o + r], t=T[:r]))
            else:
                bp, bc = builds[k]
                out.append(serve.Request(k, d["arrival"], "build", problem=bp, c=bc))
        return out

    srv = serve.Server(max_batch_rhs=args.serve_max_rhs)
    srv.add_solver("main", h)
    # warm-up: one batch and one build of each size
    warm = [serve.Request(0, 0.0, "solve", key="main", nrhs=4, s=S[:4], t=T[:4])]
    for j, (bp, bc) in enumerate({bp.m: (bp, bc) for bp, bc in builds.values()}.values()):
        warm.append(serve.Request(j + 1, 0.0, "build", problem=bp, c=bc))
    drop = lambda r: setattr(r, "u", None)  # noqa: E731  (results are not kept)
    srv.run(warm, on_done=drop)
    srv.release_built()
    torch.cuda.synchronize()
    res = {"resident_build_s": build_s, "resident_operator_bytes": h.info().operator_bytes,
           "resident_leaf_form": args.serve_resident_form, "build_leaf_form": args.leaf_form}
    backlog = srv.run(make(0.0), on_done=drop)
    srv.release_built()
    cap = serve.summarize(backlog)
    res["capacity"] = cap
    for frac in (0.5, 0.9):
        reqs = srv.run(make(frac * cap["req_per_s"]), on_done=drop)
        srv.release_built()
        res[f"load_{int(frac * 100)}"] = serve.summarize(reqs)
    h.free()
    return res


def serving(args, local_rank):
    import torch

    torch.cuda.set_device(local_rank)
    from paper_1812_07167_gb300 import hps

    out = {"metric": "HPS serving: p50/p99 request latency and throughput under Poisson load",
           "unit": "ms", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "helmholtz_serving_resident", "leaves": f"{args.serve_m}x{args.serve_m}",
                      "p": P_ORDER, "q": P_ORDER - 2, "kappa": 600.0, "eta": 600.0,
                      "c": "random medium, 32 Fourier modes, seed 3", "requests": args.serve_requests,
                      "mix": "90% solves (nrhs U{1..64}, 8 Gaussian sources, t = 0), "
                             "10% builds (m U{16,32,64}, kappa U[20,200])",
                      "max_batch_rhs": args.serve_max_rhs, "arrivals": "Poisson, seed 4"}}
    with ClockSampler(local_rank) as clk:
        out["fp64"] = serving_run(args, local_rank, hps.HPS_FP64)
        out["mixed"] = serving_run(args, local_rank, hps.HPS_MIXED)
    out["value"] = out["fp64"]["load_90"]["solve_p99_ms"]
    out["clocks"] = clk.summary()
    print(json.dumps(out), flush=True)


def profile_step(args, local_rank):
    """One bench step (build + 1-RHS solve of the 16 x 16-leaf workload) between
    cudaProfilerStart and cudaProfilerStop, after the tuner and three warm-up
    steps, for `ncu --profile-from-start off`: the profiler then sees exactly
    the kernels of one timed step, with the kernel choices the bench makes."""
    import torch

    from paper_1812_07167_gb300 import hps

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    st = torch.cuda.current_stream()
    wl = workload()
    pr = _problem(wl.m, wl.p, wl.kappa, wl.eta)
    lxy, bxy = hps.hps_nodes(pr)
    c, s, t = wl.sample(lxy, bxy)
    cd = torch.from_numpy(c).to(dev)
    sd = torch.from_numpy(np.ascontiguousarray(s[None])).to(dev)
    td = torch.from_numpy(np.ascontiguousarray(t[None])).to(dev)
    ud = torch.empty((1, pr.leaves, pr.n), dtype=torch.complex128, device=dev)
    hps.hps_tune([pr], st)
    for _ in range(3):
        h = hps.hps_build(pr, cd, st)
        hps.hps_solve(h, sd, td, ud, 1, st)
        torch.cuda.synchronize()
        h.free()
    torch.cuda.profiler.start()
    h = hps.hps_build(pr, cd, st)
    hps.hps_solve(h, sd, td, ud, 1, st)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    info = h.info()
    code = hps.hps_status(h, st)[0]
    h.free()
    print(json.dumps({"profiled_step": "16x16 build + 1-RHS solve", "status": hps.hps_strerror(code),
                      "build_launches": info.build_launches, "solve_launches": info.solve_launches}), flush=True)


def bf16_peak_sustained():
    """The measured sustained bf16 tensor rate of the GB300s
    (MEASURED_PEAKS.json), else the profiling recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["bf16_tflops_sustained"])
        return v, "measured sustained bf16 (cuBLAS loop under the power cap, MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback: sustained bf16 ~1.7 PFLOP/s (one earlier GB300 measurement)"


def stored_traffic(kernel):
    """DRAM bytes per launch from the committed ncu capture of `kernel`
    (profiles/<kernel>_traffic.json), or None once the kernel's source has
    changed since the capture."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        tr = json.load(f)
    return tr.get("bytes_per_launch") if tr.get("kernel_hash") == kernel_hash(kernel) else None


def kernel_hash(kernel="lu_leaf_kernel"):
    """Hash of the code of a leaf kernel (its file and the device headers it
    includes, comments left out), so stored ncu counters are used only for
    the code they were taken on."""
    import hashlib

    srcs = {"lu_leaf_kernel": ("lu.cu", "cx.cuh", "leaf_geom.cuh"),
            "leaf_kernel": ("gj.cu", "cx.cuh", "leaf_geom.cuh"),
            "oz_tc_kernel": ("ozaki.cu", "cx.cuh", "tc_desc.h", "hps_internal.h")}[kernel]
    h = hashlib.sha256()
    for name in srcs:
        with open(os.path.join(ROOT, "paper_1812_07167_gb300", "csrc", name)) as f:
            # the code only: // comments and blank lines do not change the kernel
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve", action="store_true", help="run the serving workload instead of the step bench")
    ap.add_argument("--precision", action="store_true",
                    help="run the 64x64-leaf FP64-vs-mixed workload (with the oracle) instead of the step bench")
    ap.add_argument("--no-batching", action="store_true", help="skip the ragged-batch section")
    ap.add_argument("--no-config3", action="store_true",
                    help="skip the 64x64-leaf kappa=300 section (FP64 and mixed, and the oracle on the host cores)")
    ap.add_argument("--polynomial", type=int, metavar="M",
                    help="capacity check: M x M leaves, polynomial solution, nodal error and memory")
    ap.add_argument("--scaling", action="store_true",
                    help="build and solve times from 4 x 4 to 128 x 128 leaves, both leaf forms")
    ap.add_argument("--leaf-form", default="inverse", choices=["lu", "inverse"],
                    help="leaf operators as B^-1 (default; a complex64 inverse refined to complex128 on the "
                         "tensor cores) or as LU factors")
    ap.add_argument("--serve-resident-form", default="inverse", choices=["lu", "inverse"],
                    help="--serve: leaf form of the resident solver (its requests are wide solves)")
    ap.add_argument("--zgemm", type=int, nargs="+", metavar="M N K [BATCH]",
                    help="time one (batched) complex GEMM on the tensor cores and on the FP64 pipes")
    ap.add_argument("--profile-step", action="store_true",
                    help="one tuned step between cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--serve-m", type=int, default=128)
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-max-rhs", type=int, default=128)
    args = ap.parse_args()
    global LEAF_FORM
    LEAF_FORM = 1 if args.leaf_form == "inverse" else 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.serve:
        serving(args, local_rank)
        return
    if args.precision:
        precision(args, local_rank)
        return
    if args.zgemm:
        zgemm(args, local_rank)
        return
    if args.profile_step:
        profile_step(args, local_rank)
        return
    if args.scaling:
        scaling(args, local_rank)
        return
    if args.polynomial:
        polynomial(args, local_rank)
        return
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    try:
        ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
