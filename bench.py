"""Benchmark of the batched lens-equation path on B300.

Headline (one JSON line on rank 0): lens evals/s (positions x components per second) of
lf_jacobian_grid in LF_MIXED precision on the cluster grid-map workload (2 elliptical dPIE
halos + 300 pseudo-Jaffe members on a 4096 x 4096 grid at 0.04", alpha, kappa, gamma, mu
at z_s = 9).  One step = one call over the whole grid (component preparation, per-pixel
sums, lens-map Jacobian and magnification in FP64).

Secondary measurements in the same line: the plain FP64 comparator on the same grid, the
batched source-plane chi^2 (4096 samples x 200 images, mixed and FP64), its gradient
(16 clusters, 22 parameters, 1024 samples), and the 3-plane ray trace (2048^2 rays).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores (bounded sample of the same
workload).  Under torchrun each rank runs the same workload (replicas; weak scaling) and
rank 0 reports the total over ranks divided by the slowest rank's time.
"""
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
sys.path.insert(0, ROOT)

METRIC = "lens evals/s (samples×positions×components)"
UNIT = "lens evals/s"
WORKLOAD = ("cluster_dpie302_grid4096: 2 elliptical dPIE halos + 300 PJE members, "
            "4096x4096 grid at 0.04\", alpha/kappa/gamma/mu at z_s=9")
# The algorithmic work of one evaluation (alpha and psi_ij of a round pseudo-Jaffe member at one
# position, the closed form of the method with its float-float offset and the accumulation):
# 33 FP32 lane operations -- offsets 6, r^2 2, S^2 and R^2 2, S and R 2, S + s and R + a 2, their
# product 1, P and Q 2, R + S 1, kbar 3, t 5, sums 7 -- and 4 MUFU operations (2 rsqrt, 2 rcp).
# The kernels may issue more or less (the anchored maps issue 36 per member for their precision;
# the chi^2 kernel's packed loop 31, its offsets leaving out the position's low word, which a
# per-image first-order term restores; the halos and folds add more): the roofline counts the
# method's work, not the implementation's, and the chi^2 line states the issued count beside it.
FP32_INSTR_PER_EVAL = 33
XU_INSTR_PER_EVAL = 4
FP32_LANES_PER_SM, XU_LANES_PER_SM = 128, 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-chi2", action="store_true", help="skip the chi^2 kernel's roofline (profiling runs)")
    ap.add_argument("--grid", type=int, default=4096)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "ff", "fp64"],
                    help="precision of the headline step")
    ap.add_argument("--workload", default="grid", choices=["grid", "chi2", "grad", "trace"],
                    help="grid = the headline; the others run one secondary kernel alone (profiling)")
    ap.add_argument("--samples", type=int, default=4096, help="samples for --workload chi2")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def max_over_ranks(x, world, device):
    """The largest value of x over the ranks: the job's step time is its slowest rank's."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reference_arm(args):
    """FP64 CPU oracle on the host cores: a seeded row band of the same grid workload."""
    import torch
    world, rank, _ = dist_init()
    if rank != 0:
        return
    from oracle import cosmology as cz
    from oracle import lensing as OL
    from oracle import model as OM
    from paper_2609_08649_b300 import workloads as W
    torch.set_num_threads(os.cpu_count() or 1)
    wl = W.cluster_c1(args.grid)
    pl = OM.build_planes(wl)[0]
    a = cz.a_dis(0.5, 9.0)
    g = wl.grid
    rows = 8
    xs = g.x0 + g.dx * np.arange(g.nx)
    times = []
    n_comp = len(pl.kind) + pl.n_members
    for step in range(args.warmup + args.steps):
        j0 = (step * 131) % (g.ny - rows)
        ys = g.y0 + g.dy * np.arange(j0, j0 + rows)
        X, Y = np.meshgrid(xs, ys)
        t0 = time.perf_counter()
        out = OL.plane_sum(pl, torch.tensor(X.ravel())[None], torch.tensor(Y.ravel())[None])
        OL.jacobian_maps(*out, a)
        t = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(t)
    evals = rows * g.nx * n_comp
    v = evals / statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64 CPU oracle",
                       "sample": f"{rows} of {g.ny} grid rows per step"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": torch.get_num_threads(),
                             "kind": "oracle", "sample": f"{rows} grid rows x {g.nx} px x {n_comp} components per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


ALPHA_TARGET = 1e-6   # arcsec: the stated deflection tolerance against the FP64 oracle


def cpu_baseline(wl, outs, prec, seconds_target=15.0):
    """The oracle as it stands on the host cores, on a bounded row band of the grid.  The rows
    it evaluates also give the headline maps' alpha error against the oracle (parity)."""
    import torch
    from oracle import cosmology as cz
    from oracle import lensing as OL
    from oracle import model as OM
    torch.set_num_threads(os.cpu_count() or 1)
    pl = OM.build_planes(wl)[0]
    a = cz.a_dis(0.5, 9.0)
    g = wl.grid
    xs = g.x0 + g.dx * np.arange(g.nx)
    n_comp = len(pl.kind) + pl.n_members
    done, t_tot, rows = 0, 0.0, 4
    j0 = g.ny // 3
    dmax, dsq = 0.0, 0.0
    while t_tot < seconds_target and done < 256:
        ys = g.y0 + g.dy * np.arange(j0 + done, j0 + done + rows)
        X, Y = np.meshgrid(xs, ys)
        t0 = time.perf_counter()
        out = OL.plane_sum(pl, torch.tensor(X.ravel())[None], torch.tensor(Y.ravel())[None])
        OL.jacobian_maps(*out, a)
        t_tot += time.perf_counter() - t0
        lo, hi = (j0 + done) * g.nx, (j0 + done + rows) * g.nx
        d = np.hypot(outs["ax"][lo:hi].cpu().numpy() - out[0][0].numpy(),
                     outs["ay"][lo:hi].cpu().numpy() - out[1][0].numpy())
        dmax, dsq = max(dmax, float(d.max())), dsq + float((d ** 2).sum())
        done += rows
    base = {"value": done * g.nx * n_comp / t_tot, "unit": UNIT, "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": f"{done} grid rows x {g.nx} px x {n_comp} components ({t_tot:.1f} s, FP64 torch CPU)"}
    parity = {"alpha_max_abs_err_arcsec": dmax, "alpha_rms_err_arcsec": (dsq / (done * g.nx)) ** 0.5,
              "pixels": done * g.nx, "rows": f"{j0}..{j0 + done - 1}", "precision": prec,
              "alpha_target_arcsec": ALPHA_TARGET, "alpha_target_met": dmax <= ALPHA_TARGET}
    return base, parity


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2609_08649_b300 import api
    from paper_2609_08649_b300 import model as PM
    from paper_2609_08649_b300 import workloads as W
    if args.workload != "grid":
        single_workload(args, torch, api, PM, W)
        return

    wl = W.cluster_c1(args.grid)
    g = wl.grid
    dp = PM.device_planes(wl)[0]
    a = PM.adis(wl.cosmo, 0.5, 9.0)
    n_pix = g.nx * g.ny
    n_comp = len(dp.comp_host) + len(dp.mem_host)
    evals = n_pix * n_comp
    outs = {k: torch.empty(n_pix, dtype=torch.float32 if k in ("kappa", "g1", "g2") else torch.float64,
                           device="cuda") for k in api.ALL_OUTPUTS}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    import ctypes as C
    from paper_2609_08649_b300 import _lib as L
    ps, gs = dp.c_struct(), PM.grid_struct(g)
    stream = torch.cuda.current_stream()

    head_prec = api.PRECISION[args.precision]

    def step(prec=head_prec):
        L.check(L.lib.lf_jacobian_grid(C.byref(ps), C.byref(gs), a, prec,
                                       *[C.c_void_p(outs[k].data_ptr()) for k in api.ALL_OUTPUTS],
                                       C.c_void_p(stream.cuda_stream)))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_region = time.perf_counter()
    for e0, e1 in evs:
        flush.fill_(1)                       # L2 flush between steps, outside the step events
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    t_region = time.perf_counter() - t_region
    clk = clocks.stop()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    ms = max_over_ranks(statistics.mean(step_ms), world, "cuda")
    value = world * evals / (ms * 1e-3)

    # end to end through the C ABI with host buffers: the plane tables host->device, then
    # lf_jacobian_grid_host (row bands computed while the previous band's maps are copied to
    # pinned host memory)
    host_out = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in outs.items()}
    comp_h = torch.from_numpy(dp.comp_host.view(np.uint8).copy()).pin_memory()
    mem_h = torch.from_numpy(dp.mem_host.view(np.uint8).copy()).pin_memory()
    h2d = comp_h.numel() + mem_h.numel()
    d2h = sum(v.numel() * v.element_size() for v in outs.values())
    ws = torch.empty(max(1, L.lib.lf_jacobian_grid_host_workspace(C.byref(gs), E2E_BANDS)), dtype=torch.uint8,
                     device="cuda")
    host_ptrs = [C.c_void_p(host_out[k].data_ptr()) for k in api.ALL_OUTPUTS]

    def step_host():
        L.check(L.lib.lf_jacobian_grid_host(C.byref(ps), C.byref(gs), a, head_prec, *host_ptrs, E2E_BANDS,
                                            C.c_void_p(ws.data_ptr()), ws.numel(), C.c_void_p(stream.cuda_stream)))

    e2e_ms = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dp.comp_dev.copy_(comp_h, non_blocking=True)
        dp.mem_dev.copy_(mem_h, non_blocking=True)
        step_host()
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_step = max_over_ranks(statistics.mean(e2e_ms), world, "cuda")
    e2e = {"value": world * evals / (e2e_step * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step,
           "call": f"lf_jacobian_grid_host, {E2E_BANDS} row bands, copies overlapped with the computation"}

    # roofline of the dominant kernel (the per-pixel sum): FP32 and XU issue against peak
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    sm_max = (clk.get("sm_max_mhz") or 2032.0) * 1e6
    fp32_peak = nsm * FP32_LANES_PER_SM * sm_max / 1e12
    xu_peak = nsm * XU_LANES_PER_SM * sm_max / 1e12
    fp32_ach = evals * FP32_INSTR_PER_EVAL / (ms * 1e-3) / 1e12
    xu_ach = evals * XU_INSTR_PER_EVAL / (ms * 1e-3) / 1e12
    traffic = map_kernel_traffic() if args.precision == "mixed" and args.grid == 4096 else None
    fma_s, fma2_s, rsq_s, dfma_s = api.probe_alu2()
    roofline = {"bound": "alu", "achieved": fp32_ach, "peak": fp32_peak, "unit": "T FP32 lane-ops/s",
                "frac": fp32_ach / fp32_peak, "traffic": traffic,
                "xu": {"achieved": xu_ach, "peak": xu_peak, "frac": xu_ach / xu_peak},
                "measured_rates": {"fp32_fma_T_per_s": fma_s / 1e12,
                                   "fp32_fma2_lane_T_per_s": fma2_s / 1e12,   # packed f32x2: same datapath
                                   "mufu_rsqrt_T_per_s": rsq_s / 1e12,
                                   "fp64_fma_T_per_s": dfma_s / 1e12,
                                   "frac_of_measured_fp32": fp32_ach / (fma_s / 1e12),
                                   "frac_of_measured_xu": xu_ach / (rsq_s / 1e12)},
                "hbm_achieved_gbs": d2h / (ms * 1e-3) / 1e9,
                "peak_source": f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max/1e6:.0f} MHz (max SM clock)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"mixed": "f32+f64", "ff": "f32x2+f64", "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": {
                "mixed": "LF_MIXED (each member's deflection at the centre of every 16x16-pixel tile in float-float "
                         "and its change across the tile in FP32; fast-changing members and the halos in "
                         "float-float; FP32 psi_ij; FP64 det/mu)",
                "ff": "LF_FF (float-float deflections of every component, FP32 psi_ij, FP64 det/mu)",
                "fp64": "LF_FP64"}[args.precision],
                       "parallelism": "replicas" if world > 1 else "1 GPU",
                       "l2": "256 MiB buffer written between timed steps, outside the step events; "
                             "each step writes 604 MB of maps (> 126 MB L2)",
                       "region_s": t_region},
            "e2e": e2e, "gpu_launches": args.steps, "clocks": clk, "roofline": roofline}

    if rank == 0 and not args.no_cpu_baseline:      # before the secondary runs reuse the map buffers
        line["cpu_baseline"], line["parity"] = cpu_baseline(wl, outs, args.precision)
    if rank == 0 and not args.no_chi2:
        line["roofline_chi2"] = chi2_roofline(torch, api, PM, W, flush, fp32_peak, xu_peak)
    if rank == 0 and not args.no_secondary:
        line["secondary"] = secondary(torch, api, PM, W, L, C, step, ms, evals)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


E2E_BANDS = 32   # row bands of the end-to-end call (each band's maps are copied while the next is computed)

KERNEL_SOURCES = ["lf_common.cuh", "lf_cse_table.h", "lf_eval.cuh", "lf_grid.cu", "lf_internal.h"]


def map_kernel_traffic():
    """DRAM bytes per launch of the headline kernel from the committed ncu capture, or None
    when the kernel's sources changed since the counters were taken."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "k_map_anchor_traffic.json")
    if not os.path.exists(prof):
        return None
    try:
        rec = json.load(open(prof))
    except ValueError:
        return None
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2609_08649_b300", "csrc", f), "rb").read())
    return rec.get("dram_bytes_per_launch") if h.hexdigest()[:16] == rec.get("source_digest") else None


def _time(torch, fn, reps=3, warm=1):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def secondary(torch, api, PM, W, L, C, step, ms_mixed, evals):
    out = {}
    ms64 = _time(torch, lambda: step(L.LF_FP64), reps=2)
    out["grid_fp64"] = {"ms": ms64, "lens_evals_per_s": evals / (ms64 * 1e-3),
                        "headline_speedup": ms64 / ms_mixed}
    msff = _time(torch, lambda: step(L.LF_FF), reps=3)
    out["grid_ff"] = {"ms": msff, "lens_evals_per_s": evals / (msff * 1e-3), "fp64_over_ff": ms64 / msff}
    # batched chi^2, 4096 samples x 200 images x 302 components
    wl = W.cluster_c2()
    cat = W.load_catalogue("cluster_200")
    th = torch.tensor(W.sample_thetas(wl, wl.seed), device="cuda")
    ev = th.shape[0] * len(cat.theta_obs) * (2 + 1 + 300)
    res = {}
    for prec in ("mixed", "ff", "fp64"):
        plan = api.Plan([PM.cluster_input(wl, cat)], th.shape[0], prec, flags=api.FLAG_GRAPH | api.FLAG_AUTOTUNE)
        t = _time(torch, lambda: plan.chi2(th), reps=5 if prec != "fp64" else 2)
        res[prec] = {"ms": t, "chi2_per_s": th.shape[0] / (t * 1e-3), "lens_evals_per_s": ev / (t * 1e-3),
                     "tile": plan.info()}
        plan.close()
    res["mixed_speedup"] = res["fp64"]["ms"] / res["mixed"]["ms"]
    res["ff_speedup"] = res["fp64"]["ms"] / res["ff"]["ms"]
    out["chi2_4096x200"] = res
    # gradient over 16 clusters
    try:
        wls = W.multicluster_c4()
        cats = [W.load_catalogue(f"multicluster_{c:02d}") for c in range(len(wls))]
        ths = np.concatenate([W.sample_thetas(w, w.seed) for w in wls])
        th4 = torch.tensor(ths, device="cuda")
        ev4 = sum(w.n_samples * len(c.theta_obs) * (3 + len(w.planes[0].members.x)) for w, c in zip(wls, cats))
        res = {}
        for prec in ("mixed", "ff", "fp64"):
            plan = api.Plan([PM.cluster_input(w, c) for w, c in zip(wls, cats)], th4.shape[0], prec,
                            flags=api.FLAG_GRAPH)
            t = _time(torch, lambda: plan.chi2_grad(th4), reps=3 if prec != "fp64" else 1)
            tc = _time(torch, lambda: plan.chi2(th4), reps=3 if prec != "fp64" else 1)
            res[prec] = {"grad_ms": t, "chi2_ms": tc, "grad_samples_per_s": th4.shape[0] / (t * 1e-3),
                         "lens_evals_per_s_chi2": ev4 / (tc * 1e-3)}
            plan.close()
        res["mixed_speedup_grad"] = res["fp64"]["grad_ms"] / res["mixed"]["grad_ms"]
        res["ff_speedup_grad"] = res["fp64"]["grad_ms"] / res["ff"]["grad_ms"]
        out["grad_16clusters_1024"] = res
    except FileNotFoundError as e:
        out["grad_16clusters_1024"] = {"skipped": str(e)}
    # total chi^2 with the flux and time-delay terms (75 magnitudes, 15 families with delays)
    aux = W.load_aux("cluster_200")
    res = {}
    for prec in ("mixed", "ff", "fp64"):
        plan = api.Plan([PM.cluster_input(wl, cat, aux=aux)], th.shape[0], prec,
                        flags=api.FLAG_GRAPH | api.FLAG_AUTOTUNE)
        t = _time(torch, lambda: plan.chi2(th), reps=5 if prec != "fp64" else 2)
        res[prec] = {"ms": t, "chi2_per_s": th.shape[0] / (t * 1e-3)}
        plan.close()
    out["chi2_flux_delay_4096x200"] = res
    # free source redshifts: 12 families' a_dis sampled as parameters (30 parameters in all)
    base_a = [PM.adis(wl.cosmo, wl.planes[0].z, z) for z in cat.fam_zs]
    fr = list(range(0, 60, 5))
    wlf = W.with_free_adis(wl, fr, [base_a[f] for f in fr], jitter=0.005)
    thf = torch.tensor(W.sample_thetas(wlf, wlf.seed), device="cuda")
    res = {}
    for prec in ("mixed", "ff"):
        plan = api.Plan([PM.cluster_input(wlf, cat)], thf.shape[0], prec, flags=api.FLAG_GRAPH | api.FLAG_AUTOTUNE)
        tc = _time(torch, lambda: plan.chi2(thf), reps=5)
        tg = _time(torch, lambda: plan.chi2_grad(thf), reps=3)
        res[prec] = {"chi2_ms": tc, "grad_ms": tg, "chi2_per_s": thf.shape[0] / (tc * 1e-3),
                     "grad_samples_per_s": thf.shape[0] / (tg * 1e-3)}
        plan.close()
    out["free_adis_4096x200_P30"] = res
    # the Hera-like model: two elliptical NFW halos (38-term CSE sums), shear, multipole,
    # 300 members; 14 parameters
    wle = W.cluster_c5_enfw()
    the = torch.tensor(W.sample_thetas(wle, wle.seed), device="cuda")
    res = {}
    for prec in ("mixed", "ff", "fp64"):
        plan = api.Plan([PM.cluster_input(wle, cat)], the.shape[0], prec, flags=api.FLAG_GRAPH | api.FLAG_AUTOTUNE)
        tc = _time(torch, lambda: plan.chi2(the), reps=5 if prec != "fp64" else 1)
        tg = _time(torch, lambda: plan.chi2_grad(the), reps=3 if prec != "fp64" else 1)
        res[prec] = {"chi2_ms": tc, "grad_ms": tg, "chi2_per_s": the.shape[0] / (tc * 1e-3),
                     "grad_samples_per_s": the.shape[0] / (tg * 1e-3)}
        plan.close()
    res["mixed_speedup_chi2"] = res["fp64"]["chi2_ms"] / res["mixed"]["chi2_ms"]
    out["chi2_enfw_4096x200"] = res
    # three lens planes: chi^2, chi^2 + gradient (the recursion's adjoint) and the image-plane
    # chi^2 (Newton with the recursion's beta and A), 1024 samples, C2's 200 image positions
    # traced to z = 4
    wl3 = W.multiplane_c3(n_grid=8)
    cat3 = W.Catalogue(cat.theta_obs, cat.theta_true, cat.fam_off, np.full(len(cat.fam_zs), 4.0))
    th3 = torch.tensor(W.sample_thetas(wl3, wl3.seed), device="cuda")
    res = {}
    for prec in ("mixed", "ff", "fp64"):
        plan = api.Plan([PM.cluster_input(wl3, cat3)], th3.shape[0], prec, flags=api.FLAG_GRAPH | api.FLAG_AUTOTUNE)
        reps = 3 if prec != "fp64" else 1
        tc = _time(torch, lambda: plan.chi2(th3), reps=reps)
        tg = _time(torch, lambda: plan.chi2_grad(th3), reps=reps)
        ti = _time(torch, lambda: plan.chi2_img(th3, iters=8), reps=reps)
        res[prec] = {"chi2_ms": tc, "grad_ms": tg, "chi2_img_ms": ti,
                     "grad_samples_per_s": th3.shape[0] / (tg * 1e-3)}
        plan.close()
    out["multiplane_3planes_1024x200"] = res
    # image-plane chi^2 (Newton model images) and the on-device sampler on the same cluster
    res = {}
    wl2 = W.cluster_c2()
    th2 = torch.tensor(W.sample_thetas(wl2, wl2.seed), device="cuda")
    for prec in ("mixed", "ff"):
        plan = api.Plan([PM.cluster_input(wl2, cat)], th2.shape[0], prec, flags=api.FLAG_AUTOTUNE)
        plan.chi2(th2)
        t = _time(torch, lambda: plan.chi2_img(th2, iters=8), reps=3)
        res[prec] = {"ms": t, "chi2_img_per_s": th2.shape[0] / (t * 1e-3), "newton_iters": 8}
        plan.close()
    out["chi2_img_4096x200"] = res
    res = {}
    sd = np.array([p.jitter * (abs(p.base) if p.relative else 1) for p in wl2.params])
    lo = torch.tensor(th2[0].cpu().numpy() - 20 * sd, device="cuda")
    hi = torch.tensor(th2[0].cpu().numpy() + 20 * sd, device="cuda")
    steps = 10
    u = torch.tensor(W.sampler_uniforms(3, steps, th2.shape[0]), device="cuda")
    for prec in ("mixed", "ff"):
        plan = api.Plan([PM.cluster_input(wl2, cat)], th2.shape[0] // 2, prec, flags=api.FLAG_AUTOTUNE)
        x = th2.clone()
        c = torch.cat([plan.chi2(x[:x.shape[0] // 2].contiguous()), plan.chi2(x[x.shape[0] // 2:].contiguous())])
        plan.aies_run(x, c, u[:1], 2.0, lo, hi)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        acc, _ = plan.aies_run(x, c, u, 2.0, lo, hi)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[prec] = {"walkers": int(x.shape[0]), "ms_per_step": ms, "steps_per_s": 1e3 / ms,
                     "chi2_per_s": x.shape[0] * 1e3 / ms, "acceptance": int(acc) / (steps * x.shape[0])}
        plan.close()
    out["aies_4096_walkers"] = res
    res = {}
    zn, un = W.mh_randoms(5, steps, th2.shape[0], th2.shape[1])
    zn, un = torch.tensor(zn, device="cuda"), torch.tensor(un, device="cuda")
    st = torch.tensor(0.3 * sd, device="cuda")
    for prec in ("mixed", "ff"):
        plan = api.Plan([PM.cluster_input(wl2, cat)], th2.shape[0], prec, flags=api.FLAG_AUTOTUNE)
        x = th2.clone()
        c = plan.chi2(x)
        plan.mh_run(x, c, zn[:1], un[:1], st, lo, hi)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        acc, _ = plan.mh_run(x, c, zn, un, st, lo, hi)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[prec] = {"chains": int(x.shape[0]), "ms_per_step": ms, "steps_per_s": 1e3 / ms,
                     "chi2_per_s": x.shape[0] * 1e3 / ms, "acceptance": int(acc) / (steps * x.shape[0])}
        plan.close()
    out["mh_4096_chains"] = res
    # lens-equation solver: 60 seeded sources (z_s of the catalogue's families) on a 1601^2
    # vertex grid over the 160" field, Newton polish in FP64
    srcs = torch.tensor(W.source_candidates(23, 60, 12.0, 4.0, -3.0), device="cuda")
    adis = torch.tensor([PM.adis(wl2.cosmo, wl2.planes[0].z, z) for z in wl2.family_zs],
                        dtype=torch.float64, device="cuda")
    fgrid = W.Grid(-80.0, -80.0, 0.1, 0.1, 1601, 1601)
    fplane = PM.device_planes(wl2)[0]
    ws = torch.empty(api.find_images_workspace(fgrid, 60, 32), dtype=torch.uint8, device="cuda")
    res = {}
    for prec in ("mixed", "fp64"):
        t = _time(torch, lambda: api.find_images(fplane, fgrid, srcs, adis, max_img=32, polish_iters=50,
                                                 precision=prec, workspace=ws), reps=3)
        _, nimg = api.find_images(fplane, fgrid, srcs, adis, max_img=32, polish_iters=50, precision=prec,
                                  workspace=ws)
        res[prec] = {"ms": t, "sources_per_s": 60 / (t * 1e-3), "images": int(nimg.clamp(min=0).sum())}
    out["find_images_60src_1601sq"] = res
    # the same solver behind three planes: 60 sources at z = 4, the 1601^2 vertex grid traced
    # through the recursion, Newton polish on the FP64 recursion
    wl3f = W.multiplane_c3(n_grid=8)
    planes3 = PM.device_planes(wl3f)
    rt = PM.multiplane_ratios(wl3f.cosmo, [p.z for p in wl3f.planes], 4.0)
    wsm = torch.empty(api.find_images_multiplane_workspace(fgrid, 60, 32), dtype=torch.uint8, device="cuda")
    res = {}
    for prec in ("mixed", "fp64"):
        t = _time(torch, lambda: api.find_images_multiplane(planes3, rt, fgrid, srcs, max_img=32, polish_iters=20,
                                                            precision=prec, workspace=wsm), reps=3)
        _, nimg = api.find_images_multiplane(planes3, rt, fgrid, srcs, max_img=32, polish_iters=20,
                                             precision=prec, workspace=wsm)
        res[prec] = {"ms": t, "sources_per_s": 60 / (t * 1e-3), "images": int(nimg.clamp(min=0).sum())}
    out["find_images_3planes_60src_1601sq"] = res
    # 3-plane trace of a 2048^2 grid
    wl3 = W.multiplane_c3()
    planes = PM.device_planes(wl3)
    r = PM.multiplane_ratios(wl3.cosmo, [p.z for p in wl3.planes], wl3.z_s)
    res = {}
    nrays = wl3.grid.nx * wl3.grid.ny
    ncomp = sum(len(p.comp_host) + len(p.mem_host) for p in planes)
    for prec in ("mixed", "ff", "fp64"):
        t = _time(torch, lambda: api.trace_multiplane(planes, r, grid=wl3.grid, precision=prec), reps=2)
        res[prec] = {"ms": t, "rays_per_s": nrays / (t * 1e-3), "lens_evals_per_s": nrays * ncomp / (t * 1e-3)}
    res["mixed_speedup"] = res["fp64"]["ms"] / res["mixed"]["ms"]
    out["trace_3plane_2048"] = res
    api.device_error()
    return out


def chi2_roofline(torch, api, PM, W, flush, fp32_peak, xu_peak, reps=10):
    """lf_chi2_batch (mixed, 4096 samples x 200 images x 303 components, graph + tuned tile)
    against the FP32 and XU issue peaks at the method's per-evaluation work, each launch timed
    alone on the launching stream after an L2 flush; and its speed-up over the FP64 kernel."""
    wl = W.cluster_c2()
    cat = W.load_catalogue("cluster_200")
    th = torch.tensor(W.sample_thetas(wl, wl.seed), device="cuda")
    n_comp = 2 + 1 + len(wl.planes[0].members.x)
    evals = th.shape[0] * len(cat.theta_obs) * n_comp
    stream = torch.cuda.current_stream()
    res, vals = {}, {}
    for prec, n in (("mixed", reps), ("fp64", 2)):
        plan = api.Plan([PM.cluster_input(wl, cat)], th.shape[0], prec, flags=api.FLAG_GRAPH | api.FLAG_AUTOTUNE)
        for _ in range(3):
            vals[prec] = plan.chi2(th).cpu().numpy()
        ts = []
        for _ in range(n):
            flush.fill_(2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.chi2(th)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        res[prec] = statistics.median(ts)
        plan.close()
    t = res["mixed"] * 1e-3
    fp32 = evals * FP32_INSTR_PER_EVAL / t / 1e12
    xu = evals * XU_INSTR_PER_EVAL / t / 1e12
    # every sample of the launch against the FP64 kernel (itself within 1e-10 of the oracle)
    rel = np.abs(vals["mixed"] - vals["fp64"]) / np.abs(vals["fp64"])
    return {"kernel": "k_chi2<LF_MIXED> (lf_chi2_batch)", "bound": "alu", "achieved": fp32, "peak": fp32_peak,
            "unit": "T FP32 lane-ops/s", "frac": fp32 / fp32_peak,
            "xu": {"achieved": xu, "peak": xu_peak, "frac": xu / xu_peak},
            "ms": res["mixed"], "fp64_ms": res["fp64"], "speedup_vs_fp64": res["fp64"] / res["mixed"],
            "chi2_per_s": th.shape[0] / t, "evals_per_launch": evals,
            "issued_fp32_per_member": 31,
            "chi2_vs_fp64_kernel": {"max_rel": float(rel.max()), "samples": int(rel.size),
                                    "over_1e-5": int((rel > 1e-5).sum()), "target_rel": 1e-5},
            "workload": f"{th.shape[0]} samples x {len(cat.theta_obs)} images x {n_comp} components"}


def single_workload(args, torch, api, PM, W):
    """One secondary kernel alone, for profiling (prints a short JSON line)."""
    prec = args.precision
    if args.workload in ("chi2", "grad"):
        wl = W.cluster_c2(n_samples=args.samples)
        cat = W.load_catalogue("cluster_200")
        th = torch.tensor(W.sample_thetas(wl, wl.seed), device="cuda")
        plan = api.Plan([PM.cluster_input(wl, cat)], th.shape[0], prec, flags=api.FLAG_AUTOTUNE)
        plan.chi2(th)   # tunes the tile shape once
        fn = (lambda: plan.chi2(th)) if args.workload == "chi2" else (lambda: plan.chi2_grad(th))
        info = plan.info()
    else:
        wl3 = W.multiplane_c3(n_grid=args.grid // 2)
        planes = PM.device_planes(wl3)
        r = PM.multiplane_ratios(wl3.cosmo, [p.z for p in wl3.planes], wl3.z_s)
        fn = lambda: api.trace_multiplane(planes, r, grid=wl3.grid, precision=prec)
        info = {}
    for _ in range(args.warmup):
        fn()
    ms = _time(torch, fn, reps=args.steps, warm=0)
    print(json.dumps({"workload": args.workload, "precision": prec, "ms": ms, "tile": info}), flush=True)


if __name__ == "__main__":
    main()
