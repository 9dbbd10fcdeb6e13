"""Benchmark: G_pq(w) points per second of the MOR-accelerated, mixed-precision IP-GFCC pipeline.

One step = the whole hot path on one synthetic molecule-sized problem, through the C ABI:
  gfcc_init (H-bar build on the GPU) -> gfcc_mor_build (batched GMRES-IR solves at the seed
  frequencies, orthonormalisation, projection) -> gfcc_mor_refine (adaptive midpoint refinement to
  the reduced-residual tolerance) -> gfcc_mor_eval (G_pq and A on the dense output grid).
value = N_w * N_p / step time (G points per second, p = q = occupied spin-orbitals).

Default workload: benzene-sized, o = 42 occupied and v = 186 virtual spin-orbitals (D = 160,188),
5000 output frequencies on [-1.0, -0.2] Ha, eta = 0.01, 8 seed frequencies, reduced-residual
tolerance 1e-6, solver tolerance 1e-8, inner sigma in TF32 on the tensor cores.

--impl reference times the FP64 CPU oracle (full-dimension GMRES solves for a bounded sample of
(w, p) points at the same size) on the host cores and prints the same kind of line.
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
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "G_pq(w) points/s, MOR + mixed precision"
METRIC_EA = "G^EA_pq(w) points/s (electron-attachment half), MOR + mixed precision"
UNIT = "points/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="benzene_o42_v186", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", default="tf32", choices=["tf32", "bf16", "fp64"])
    ap.add_argument("--nomega", type=int, default=0, help="output grid size (0: the workload's)")
    ap.add_argument("--seeds", type=int, default=8)
    ap.add_argument("--mor-tol", type=float, default=1e-6)
    ap.add_argument("--ngrid", type=int, default=500, help="refinement check grid")
    ap.add_argument("--m-max", type=int, default=1700)
    ap.add_argument("--solve-tol", type=float, default=1e-8)
    ap.add_argument("--restart", type=int, default=30, help="GMRES(k) Krylov dimension per cycle")
    ap.add_argument("--siso", action="store_true",
                    help="one reduced model of G_pp per orbital (gfcc_mor_build_siso) instead of one MIMO model")
    ap.add_argument("--pset", default="", choices=["", "occupied", "all"],
                    help="orbital set p (= q set): the workload's default, the occupied or all spin-orbitals")
    ap.add_argument("--krylov", type=int, default=0,
                    help="K > 0: reduced model on the block Krylov space of M on the b_p (gfcc_mor_build_krylov, K "
                         "initial blocks, grown by the refinement) instead of solutions at sampled frequencies")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="timed end-to-end steps through host buffers (at most --steps), after one warm-up step")
    ap.add_argument("--full-stride", type=int, default=50,
                    help="every k-th output frequency, plus the sampled ones and the middle of the window, is also "
                         "solved full-dimension in FP64 for comparison (0: skip)")
    ap.add_argument("--cpu-sample", type=int, default=1, help="(w, p) columns in the oracle sample")
    ap.add_argument("--ref-iters", type=int, default=6,
                    help="--impl reference: GMRES iterations of the oracle per timed step")
    ap.add_argument("--model-only", action="store_true",
                    help="--mode autograd: only the derivative-driven reduced model (no gradient checks)")
    ap.add_argument("--max-batch", type=int, default=0,
                    help="--mode autograd: largest batch of columns per solve in the reduced-model step (0: from memory)")
    ap.add_argument("--mode", default="pipeline", choices=["pipeline", "sigma", "peaks", "autograd"],
                    help="pipeline: the whole MOR step (default); sigma: one batch of sigma applications; "
                         "peaks: FP64, TF32 and BF16 GEMM rates of this GPU (library GEMMs, timing only); "
                         "autograd: gradients by the adjoint solves against finite differences, and the "
                         "derivative-driven reduced model (run it with --workload adenine_o70_v250)")
    ap.add_argument("--nvec", type=int, default=64, help="vectors per sigma batch (--mode sigma)")
    ap.add_argument("--sector", default="ip", choices=["ip", "ea"],
                    help="ip: the ionisation half (1h + 2h1p, default); ea: the electron-attachment half "
                         "(1p + 2p1h space, gfcc_init_ea) on the workload's attachment window, p = q = the "
                         "min(o, v) lowest virtual spin-orbitals (all spin-orbitals where the workload uses all)")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum, averaged over the captured launches) of
# the roofline kernel, from an ncu capture of the same kernel; valid only while the kernel's source file
# is unchanged (its SHA-256 is recorded with the figure).
TRAFFIC = {
    ("benzene_o42_v186", 11): {
        "bytes_per_launch": 5.168e9,
        "tc_gemm_sha256": "9110833ea70b31ddbac7b19b06fd3679fe50bf183f47b00561481f78df21f98e",
        "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum over the 175 ring-GEMM launches of a timed "
                  "benchmark step (NVTX range gfcc_ring_gemm, one pass), averaged",
    },
}


def _sha256(path):
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def measured_traffic(workload, cls):
    t = TRAFFIC.get((workload, cls))
    if not t:
        return None
    src = os.path.join(ROOT, "paper_1902_06016_gb300", "csrc", "tc_gemm.cu")
    return t if os.path.exists(src) and _sha256(src) == t["tc_gemm_sha256"] else None


# Dense GEMM rates measured on a GB300 of this machine with `python bench.py --mode peaks` (cuBLAS through
# torch.matmul, 8192^3, CUDA events, SM clock 2070 MHz, sw_power_cap only): the TF32 and FP64 rates that
# the driver does not measure. The roofline's `peak` for a TF32 contraction follows the rule "measured
# bf16 x the nominal tf32/bf16 ratio (1.1 / 2.25 PFLOP/s)"; these figures are reported beside it.
OWN_PEAKS = {"tf32_tflops": 1008.3, "tf32_tflops_sustained": 897.0, "fp64_tflops": 1.099,
             "bf16_tflops": 1871.5, "bf16_tflops_sustained": 1678.3}
TF32_OVER_BF16 = 1.1 / 2.25


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------------------------
# p set of each workload (q set = p set): the occupied spin-orbitals, or all spin-orbitals where the
# workload's configuration asks for every orbital
P_SET = {"co_o14_v42": "all"}


def orbital_set(workload, o, n):
    return list(range(n)) if P_SET.get(workload) == "all" else list(range(o))


def ea_orbital_set(workload, inp):
    """p = q set of the attachment runs: all spin-orbitals where the workload uses all, else the
    min(o, v) virtual spin-orbitals of lowest energy (the attachment analogue of the occupied set)."""
    o, v = inp.o, inp.v
    if P_SET.get(workload) == "all":
        return list(range(o + v))
    k = min(o, v)
    return sorted(int(o + a) for a in np.argsort(inp.eps[o:], kind="stable")[:k])


def window(args, W):
    """(wmin, wmax) of the run: the workload's ionisation window, or its attachment window."""
    return (W["ea_wmin"], W["ea_wmax"]) if args.sector == "ea" else (W["wmin"], W["wmax"])


def pinned_copy(arr):
    """Page-locked host copy of a NumPy array (returned as a NumPy view of a pinned torch tensor)."""
    import torch
    t = torch.empty(arr.shape, dtype=torch.from_numpy(arr[:0].copy()).dtype, pin_memory=True)
    view = t.numpy()
    view[...] = arr
    return view, t


def pinned_empty(shape, dtype):
    import torch
    t = torch.empty(shape, dtype=dtype, pin_memory=True)
    return t.numpy(), t


def spectrum_peaks(A, grid, rel=0.01, sign=-1.0):
    """Peaks of the spectral function on the output grid. For the ionisation half A = -(1/pi) sum Im G_pp
    is negative at poles (the -i eta convention), so the peaks are local minima of A deeper than
    rel * max |A| (sign = -1); the attachment half (+ i eta) has positive peaks (sign = +1)."""
    a = sign * np.asarray(A)
    thr = rel * np.abs(a).max()
    k = np.where((a[1:-1] > a[:-2]) & (a[1:-1] >= a[2:]) & (a[1:-1] > thr))[0] + 1
    return {"count": int(len(k)), "threshold_rel": rel, "positions_ha": [round(float(grid[i]), 5) for i in k[:40]]}


def autotune_summary(decisions):
    """Condensed autotuner report: bucket counts, the time the chosen group sizes save over the default
    (one launch per bucket, as tuned), and the decisions for the low-precision (inner sigma) GEMMs."""
    changed = [d for d in decisions if d["gm"] != d["gm_default"]]
    return {"buckets": len(decisions), "changed_from_default": len(changed),
            "tuned_ms_sum": round(sum(d["ms_best"] for d in decisions), 3),
            "default_ms_sum": round(sum(d["ms_default"] for d in decisions), 3),
            "inner_sigma_gemms": [d for d in decisions if not d["exact_slices"]]}


def run_ours(args, rank, world):
    import torch
    from paper_1902_06016_gb300 import Context, load
    from paper_1902_06016_gb300 import gfcc as G

    dev = torch.device("cuda", rank % torch.cuda.device_count())
    torch.cuda.set_device(dev)
    load()
    W = synth.WORKLOADS[args.workload]
    o, v, eta = W["o"], W["v"], W["eta"]
    nw = args.nomega or W["nw"]
    inp = synth.make_inputs(o, v, rank_seed(W["seed"], rank))   # weak scaling: one problem per rank
    ea = args.sector == "ea"
    if ea:
        porb = list(range(o + v)) if args.pset == "all" else ea_orbital_set(args.workload, inp)
    else:
        porb = list(range(o + v)) if args.pset == "all" else (list(range(o)) if args.pset == "occupied"
                                                               else orbital_set(args.workload, o, o + v))
    npp = len(porb)
    wmin, wmax = window(args, W)
    seeds = synth.omega_grid(wmin, wmax, args.seeds)
    grid = np.linspace(wmin, wmax, nw)
    t_vvvv = None
    vp_host = vp_dev = None
    if ea:   # the packed virtual block <ab||cd> that the attachment space needs (generated once, untimed)
        t_vvvv = time.perf_counter()
        vp_host = inp.vvvv_pairs()
        t_vvvv = time.perf_counter() - t_vvvv

    # device-resident inputs (HBM) for the device-timed value
    dev_inputs = synth.Inputs(**{k: (torch.from_numpy(np.ascontiguousarray(getattr(inp, k))).to(dev)
                                     if isinstance(getattr(inp, k), np.ndarray) else getattr(inp, k))
                                 for k in inp.__dataclass_fields__})
    if ea:
        vp_dev = torch.from_numpy(vp_host).to(dev)
    G_dev = torch.empty((nw, npp, npp), dtype=torch.complex128, device=dev)
    A_dev = torch.empty((nw,), dtype=torch.float64, device=dev)
    omega_host = np.ascontiguousarray(grid)

    stream = torch.cuda.current_stream(dev)

    def step(inputs, G_out, A_out, keep=False, vvvv=None):
        ctx = Context(inputs, tol=args.solve_tol, precision=args.precision, stream=stream.cuda_stream,
                      restart=args.restart, sector=args.sector, vvvv=vvvv)
        if args.siso:
            ctx.mor_build_siso(seeds, eta, porb)
        elif args.krylov > 0:
            ctx.mor_build_krylov(args.krylov, eta, porb)
        else:
            ctx.mor_build(seeds, eta, porb)
        ref = ctx.mor_refine(wmin, wmax, args.ngrid, args.mor_tol, args.m_max)
        ctx.mor_eval(omega_host, G=G_out, A=A_out)
        info = ctx.mor_info()
        info.update(ctx.mor_stats())
        if keep:
            return ref, info, ctx
        ctx.close()
        return ref, info, None

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step(dev_inputs, G_dev, A_dev, vvvv=vp_dev)
    torch.cuda.synchronize()

    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    G.profile(True)
    l0 = G.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        ref, info, _ = step(dev_inputs, G_dev, A_dev, vvvv=vp_dev)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = G.launch_count() - l0
    dev_ms = ev0.elapsed_time(ev1) / args.steps
    classes = {k: G.profile_read(k) for k in (0, 1, 2, 11)}   # (launches, ms, flops)
    phase_names = {3: "sigma_lowprec", 4: "sigma_fp64_accurate", 5: "krylov_arnoldi", 6: "mor_orthonormalise",
                   7: "mor_eval", 8: "hbar_build", 9: "mor_panel_columns", 10: "mor_residual_basis",
                   12: "exact_slice_complex_gemms", 13: "exact_slicing", 19: "eval_hessenberg_reduction",
                   20: "eval_shifted_solves", 21: "ortho_gram_products", 22: "ortho_updates",
                   23: "ortho_panel_cholqr", 24: "exact_slice_accumulate", 25: "lowprec_operand_prep",
                   26: "lowprec_combine", 27: "input_upload", 28: "output_copies"}
    phases = {phase_names[k]: round(G.profile_read(k)[1] / args.steps, 1) for k in phase_names}
    allocs = {"allocations": G.profile_read(29)[0] // args.steps, "alloc_host_ms": round(G.profile_read(29)[1] / args.steps, 1),
              "frees": G.profile_read(30)[0] // args.steps, "free_host_ms": round(G.profile_read(30)[1] / args.steps, 1)}
    cgs = G.profile_read(14)   # (launch groups, ms, algorithmic bytes) of the Arnoldi sweeps
    slicing, accum = G.profile_read(13), G.profile_read(24)   # exact-slice passes (bytes in the third field)
    small_gemms = G.profile_read(31)   # up, oooo, down GEMMs of the low-precision sigma (bytes)
    sig_lp, sig_ex = G.profile_read(3), G.profile_read(4)      # whole sigmas (algorithmic flops)
    cgs_parts = {name: G.profile_read(k) for k, name in
                 ((15, "multidot_kernel"), (16, "cgs_update_kernel<dot>"), (17, "cgs_update_kernel<norm>"),
                  (18, "all three, batches < 32 columns"))}
    G.profile(False)
    clk = clocks.stop()
    spectrum = spectrum_peaks(A_dev.cpu().numpy(), grid, sign=1.0 if ea else -1.0)
    tuned = autotune_summary(G.autotune_report())

    # end to end through the public API with host buffers: the inputs are copied from page-locked host
    # memory inside gfcc_init and G, A are written to page-locked host arrays, every step; one warm-up
    # step, then the median of e2e_steps timed steps (wall clock around each, device synchronised)
    e2e = None
    kept = None
    if not args.no_e2e:
        keep_alive = []
        host_fields = {}
        for k in inp.__dataclass_fields__:
            a = getattr(inp, k)
            if isinstance(a, np.ndarray):
                view, t = pinned_copy(np.ascontiguousarray(a))
                keep_alive.append(t)
                host_fields[k] = view
            else:
                host_fields[k] = a
        host_inputs = synth.Inputs(**host_fields)
        vp_pinned = None
        if ea:
            vp_pinned, tv = pinned_copy(vp_host)
            keep_alive.append(tv)
        G_host, tg = pinned_empty((nw, npp, npp), torch.complex128)
        A_host, ta = pinned_empty((nw,), torch.float64)
        keep_alive += [tg, ta]
        n_e2e = max(1, min(args.steps, args.e2e_steps))
        step(host_inputs, G_host, A_host, vvvv=vp_pinned)
        torch.cuda.synchronize()
        times = []
        G.profile(True)
        for k in range(n_e2e):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, _, kc = step(host_inputs, G_host, A_host, keep=(k == n_e2e - 1), vvvv=vp_pinned)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            if kc is not None:
                kept = kc
        e2e_phases = {"input_upload": G.profile_read(27)[1] / n_e2e, "output_copies": G.profile_read(28)[1] / n_e2e,
                      "hbar_build": G.profile_read(8)[1] / n_e2e, "alloc_host": G.profile_read(29)[1] / n_e2e,
                      "free_host": G.profile_read(30)[1] / n_e2e}
        G.profile(False)
        e2e_s = statistics.median(times)
        h2d = sum(getattr(inp, k).nbytes for k in ("eps", "oooo", "ooov", "oovv", "ovov", "ovvv", "t1", "t2", "l1", "l2"))
        if ea:
            h2d += vp_host.nbytes
        e2e = {"value": nw * npp / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(G_host.nbytes + A_host.nbytes), "steps": n_e2e, "warmup": 1,
               "median_s": e2e_s, "min_s": min(times), "max_s": max(times),
               "host_memory": "page-locked (pinned) input and output arrays",
               "phases_ms": {k: round(val, 1) for k, val in e2e_phases.items()},
               "h2d_gbs": h2d / (e2e_phases["input_upload"] / 1e3) / 1e9 if e2e_phases["input_upload"] > 0 else None}
        if kept is not None:
            e2e["G_matches_device_run"] = bool(np.array_equal(G_host, G_dev.cpu().numpy()))

    # untimed by the line's value: full-dimension FP64-accurate solves at a stratified subset of the output
    # grid (every full_stride-th point), at every sampled frequency and at the oracle sample's frequency;
    # their own rate, and the reduced model's A and G errors against them
    full = None
    if args.full_stride > 0 and rank == 0:
        if kept is None:
            _, _, kept = step(dev_inputs, G_dev, A_dev, keep=True, vvvv=vp_dev)
        full = full_compare(args, kept, grid, porb, eta, stream)
    if kept is not None:
        kept.close()

    # max over ranks; every rank solved its own problem (weak scaling)
    dev_ms = max_over_ranks(dev_ms, dev, world)
    value = job_value(nw, npp, world, dev_ms)

    peaks, peak_kind = measured_peaks()
    bf16 = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    names = {0: f"tc_gemm_kernel<{args.precision}> (inner low-precision sigma GEMMs: up, oooo, down)",
             1: "gemm_kernel<double> (FP64 SIMT GEMM)",
             2: "tc_gemm_kernel<bf16, exact> on exact slices (FP64-accurate residual / projection GEMMs)",
             11: f"tc_gemm_kernel<{args.precision}> ring-term GEMM of the inner sigma"}
    ratio0 = TF32_OVER_BF16 if args.precision == "tf32" else 1.0
    kernels = {}
    for k, (n, ms, fl) in classes.items():
        if n == 0 or ms <= 0:
            continue
        ach = fl / (ms / 1e3) / 1e12
        if k == 1:
            kernels[names[k]] = {"bound": "alu", "launches": n, "ms": ms, "achieved": ach, "unit": "TFLOP/s",
                                 "peak": OWN_PEAKS["fp64_tflops"], "frac": ach / OWN_PEAKS["fp64_tflops"],
                                 "peak_kind": "FP64 DGEMM rate measured with --mode peaks (cuBLAS)"}
        else:
            pk = bf16 * (ratio0 if k in (0, 11) else 1.0)
            kernels[names[k]] = {"bound": "tensor", "launches": n, "ms": ms, "achieved": ach, "peak": pk,
                                 "unit": "TFLOP/s", "frac": ach / pk}
    roof = None
    # the roofline kernel: the ring-term GEMM (the largest single GEMM of the hot path), else the
    # tensor-core class with the most time
    dom = 11 if classes[11][0] > 0 else max((k for k in classes if classes[k][0] > 0 and k != 1),
                                            key=lambda k: classes[k][1], default=None)
    if dom is not None:
        n, ms, fl = classes[dom]
        ach = fl / (ms / 1e3) / 1e12
        pk = bf16 * (ratio0 if dom in (0, 11) else 1.0)
        tr = measured_traffic(args.workload, dom)
        roof = {"kernel": names[dom], "bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "traffic": tr["bytes_per_launch"] if tr else None,
                "traffic_source": tr["source"] if tr else "no ncu capture of the current kernel source",
                "peak_kind": f"{peak_kind} sustained bf16" + (f" x {ratio0:.4f} (nominal tf32/bf16 ratio)"
                                                              if dom in (0, 11) and ratio0 != 1 else ""),
                "launches": n, "avg_launch_ms": ms / n, "flops_per_launch": fl / n}
        if dom in (0, 11) and args.precision == "tf32":
            roof["frac_of_measured_tf32_sustained"] = ach / OWN_PEAKS["tf32_tflops_sustained"]
    return inp, {
        "metric": METRIC_EA if ea else METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dev_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"c128 (f64 residuals, {args.precision} tensor-core inner sigma)", "data": "synthetic",
        "config": {"workload": args.workload, "o": o, "v": v, "D": v + v * (v - 1) // 2 * o if ea else inp.dim,
                   "n_omega": nw, "n_p": npp, "n_q": npp,
                   **({"vvvv_generation_s": round(t_vvvv, 1)} if ea else {}),
                   "p_set": "all spin-orbitals" if npp == o + v else (
                       f"the {npp} lowest virtual spin-orbitals" if ea else "occupied spin-orbitals"),
                   "sector": "EA (1p + 2p1h, gfcc_init_ea)" if ea else "IP (1h + 2h1p)",
                   "eta": eta, "window_ha": [wmin, wmax], "seeds": args.seeds, "mor_tol": args.mor_tol,
                   "solve_tol": args.solve_tol, "restart": args.restart,
                   "reduced_model": "one SISO model of G_pp per orbital" if args.siso else
                   (f"block Krylov space of M on the b_p ({args.krylov} initial blocks)" if args.krylov > 0 else
                    "one MIMO model"),
                   "model_order": info["m"],
                   "sampled_freqs": len(info["sampled"]),
                   "arnoldi_steps": info["arnoldi_steps"], "columns_solved": info["columns"],
                   "l2": "working set (operators >= 0.5 GB, Krylov bases) larger than L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "e2e": e2e, "gpu_launches": int(launches), "gpu_launches_per_step": int(launches // args.steps),
        "roofline": roof, "gemm_classes": kernels, "phases_ms": phases, "device_allocations_per_step": allocs,
        "hbm_kernels": {"arnoldi_cgs_sweeps (multidot_kernel, cgs_update_kernel x2)": {
            "bound": "hbm", "steps": cgs[0], "ms": cgs[1], "algorithmic_bytes": cgs[2],
            "achieved": cgs[2] / (cgs[1] / 1e3) / 1e9 if cgs[1] > 0 else None, "unit": "GB/s",
            "peak": peaks.get("hbm_gbs"), "frac": (cgs[2] / (cgs[1] / 1e3) / 1e9) / peaks["hbm_gbs"]
            if cgs[1] > 0 and peaks.get("hbm_gbs") else None,
            "parts": {name: {"launches": n, "ms": round(ms, 2), "achieved_gbs": round(b / (ms / 1e3) / 1e9, 1)
                             if ms > 0 else None} for name, (n, ms, b) in cgs_parts.items()}},
            **{name: {"bound": "hbm", "launches": n, "ms": ms, "algorithmic_bytes": b, "unit": "GB/s",
                      "achieved": b / (ms / 1e3) / 1e9 if ms > 0 else None, "peak": peaks.get("hbm_gbs"),
                      "frac": b / (ms / 1e3) / 1e9 / peaks["hbm_gbs"] if ms > 0 and peaks.get("hbm_gbs") else None}
               for name, (n, ms, b) in (("exact_slicing (FP64 rows -> bf16 integer slices)", slicing),
                                        ("exact_slice_accumulate (int32 split sums -> FP64 output)", accum),
                                        (f"tc_gemm_kernel<{args.precision}> up, oooo, down GEMMs of the inner sigma "
                                         "(short or thin shapes: operands read once, outputs written once)",
                                         small_gemms))}},
        "sigma_rates": {
            "what": "the method's sigma flops (2 per multiply-add of the ring, oooo, three-body and coupling terms) "
                    "per second of the whole sigma (operand preparation, GEMMs, combine)",
            f"{args.precision}_inner": {"calls": sig_lp[0], "ms": sig_lp[1],
                                        "tflops": sig_lp[2] / (sig_lp[1] / 1e3) / 1e12 if sig_lp[1] > 0 else None},
            "fp64_accurate_exact_slices": {
                "calls": sig_ex[0], "ms": sig_ex[1],
                "fp64_equivalent_tflops": sig_ex[2] / (sig_ex[1] / 1e3) / 1e12 if sig_ex[1] > 0 else None,
                "vs_measured_fp64_rate": (sig_ex[2] / (sig_ex[1] / 1e3) / 1e12) / OWN_PEAKS["fp64_tflops"]
                if sig_ex[1] > 0 else None}},
        "clocks": clk,
        "spectrum": spectrum,
        "autotune": {"enabled": os.environ.get("GFCC_AUTOTUNE", "1") != "0",
                     "what": "M-tile group size of the tcgen05 GEMM per shape bucket, timed on first use",
                     **tuned},
        "full_fp64": full,
    }


def max_over_ranks(x: float, device, world: int) -> float:
    """The largest x over the ranks of the process group (x itself for a single process)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_omega: int, n_p: int, world: int, ms_per_step: float) -> float:
    """Whole-job G points/s: every rank evaluates n_omega x n_p points of its own problem per step."""
    return world * n_omega * n_p / (ms_per_step / 1e3)


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of the synthetic problem of a rank (independent replicas)."""
    return base_seed + rank


def full_compare(args, ctx, grid, porb, eta, stream):
    """Full-dimension FP64-accurate GMRES-IR solves (inner and residual sigma on exact bf16 slices) at every
    full_stride-th frequency of the output grid, at every frequency the reduced model sampled and at the
    middle of the window; returns their G points/s and the reduced model's A and G errors against them
    (normwise relative: max over the subset of |error| / max |full|)."""
    import torch
    W = synth.WORKLOADS[args.workload]
    nw = len(grid)
    w_grid = grid[::args.full_stride]
    sampled = np.asarray(ctx.mor_info()["sampled"])
    wlo, whi = window(args, W)
    w_mid = 0.5 * (wlo + whi)
    sub = np.concatenate([w_grid, sampled, [w_mid]])
    ng, ns = len(w_grid), len(sampled)
    ctx.set_opts(tol=args.solve_tol, precision="fp64_tc")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = ctx.solve_full(sub, eta, porb)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    mor = ctx.mor_eval(sub)
    Af, Gf = r["A"], r["G"]
    st = r["stats"]
    if args.siso:   # per-orbital models give the diagonal G_pp only: compare those
        Gf = np.diagonal(Gf, axis1=1, axis2=2)[:, :, None]
        mor = dict(mor, G=np.diagonal(mor["G"], axis1=1, axis2=2)[:, :, None])

    def err(a, b):
        return float(np.abs(a - b).max() / np.abs(b).max())

    return {"value": len(sub) * len(porb) / (ms / 1e3), "unit": UNIT, "ms": ms, "n_omega": int(len(sub)),
            "n_p": len(porb), "solver": "GMRES-IR, FP64-accurate inner and residual sigma (exact bf16 slices)",
            "converged": bool(r["converged"]), "max_rel_res": st.max_rel_res, "gmres_iters": st.gmres_iters,
            "mor_A_rel_err": err(mor["A"][:ng], Af[:ng]), "mor_G_rel_err": err(mor["G"][:ng], Gf[:ng]),
            "mor_A_rel_err_at_samples": err(mor["A"][ng:ng + ns], Af[ng:ng + ns]) if ns else None,
            "mor_G_rel_err_at_samples": err(mor["G"][ng:ng + ns], Gf[ng:ng + ns]) if ns else None,
            "omegas": f"{ng} points (every {args.full_stride}-th of the {nw}-point output grid), the {ns} sampled "
                      f"frequencies and w = {w_mid:.2f} Ha",
            "_G_mid": Gf[-1], "_G_mor_mid": mor["G"][-1]}


# ---------------------------------------------------------------------------------------------
def run_sigma(args):
    """Micro-benchmark of the dominant kernels: the sigma on one batch of nvec complex vectors."""
    import torch
    from paper_1902_06016_gb300 import Context, load
    from paper_1902_06016_gb300 import gfcc as G
    torch.cuda.set_device(0)
    load()
    W = synth.WORKLOADS[args.workload]
    inp = synth.make_inputs(W["o"], W["v"], W["seed"])
    stream = torch.cuda.current_stream()
    ctx = Context(inp, precision=args.precision, stream=stream.cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn((args.nvec, ctx.D), dtype=torch.complex128, device="cuda", generator=g)
    Y = torch.empty_like(X)
    for _ in range(args.warmup):
        ctx.sigma(X, precision=args.precision, out=Y)
    torch.cuda.synchronize()
    G.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.sigma(X, precision=args.precision, out=Y)
    e1.record(stream)
    torch.cuda.synchronize()
    n, ms, fl = G.profile_read(11 if args.precision in ("tf32", "bf16") else 2)
    n0, ms0, fl0 = G.profile_read(0)
    G.profile(False)
    o, v = W["o"], W["v"]
    P = o * (o - 1) // 2
    flop = 2.0 * args.nvec * (2 * (o * v) ** 2 * o + 2 * P * P * v + 4 * P * v * v + 4 * o * P * v)
    step_ms = e0.elapsed_time(e1) / args.steps
    peaks, kind = measured_peaks()
    bf16 = peaks.get("bf16_tflops", 1900.0)
    pk = bf16 * (TF32_OVER_BF16 if args.precision == "tf32" else 1.0)
    ach = fl / (ms / 1e3) / 1e12 if ms else None
    return {"metric": "sigma complex columns/s", "value": args.nvec / (step_ms / 1e3), "unit": "columns/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": args.workload, "nvec": args.nvec, "mode": "sigma"},
            "algorithmic_tflops": flop / (step_ms / 1e3) / 1e12,
            "roofline": {"kernel": "tc_gemm_kernel ring-term GEMM", "bound": "tensor", "achieved": ach, "peak": pk,
                         "unit": "TFLOP/s", "frac": ach / pk if ach else None, "peak_kind": f"{kind} burst bf16" +
                         (" x 1.1/2.25 (nominal tf32/bf16 ratio)" if args.precision == "tf32" else ""), "launches": n,
                         "avg_launch_ms": ms / n if n else None},
            "other_gemms": {"launches": n0, "ms": ms0,
                            "achieved": fl0 / (ms0 / 1e3) / 1e12 if ms0 else None}}


def run_peaks(args):
    """Dense GEMM rates of this GPU for the roofline denominators the driver does not measure: FP64 and
    TF32 (and BF16 for comparison with the driver's figure), square GEMMs through torch.matmul (cuBLAS),
    CUDA events on the launching stream; burst = best of 10, sustained = back to back for about 3 s."""
    import torch
    torch.cuda.set_device(0)
    out = {"metric": "dense GEMM rate", "unit": "TFLOP/s", "mode": "peaks", "kernels": "cuBLAS via torch.matmul"}
    clocks = ClockSampler(0)
    clocks.start()
    for name, dt, n, tf32 in (("fp64", torch.float64, 8192, False), ("tf32", torch.float32, 8192, True),
                              ("bf16", torch.bfloat16, 8192, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn((n, n), device="cuda").to(dt)
        b = torch.randn((n, n), device="cuda").to(dt)
        c = torch.empty((n, n), device="cuda", dtype=dt)
        for _ in range(3):
            torch.matmul(a, b, out=c)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        reps = max(3, int(3000.0 / best))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        fl = 2.0 * n ** 3
        out[name] = {"n": n, "burst_tflops": fl / (best / 1e3) / 1e12,
                     "sustained_tflops": fl * reps / (e0.elapsed_time(e1) / 1e3) / 1e12, "reps": reps}
        del a, b, c
    torch.backends.cuda.matmul.allow_tf32 = False
    out["clocks"] = clocks.stop()
    return out


def run_autograd(args):
    """Differentiation at size (default: the adenine-sized workload, o = 70, v = 250, D = 603,820).

    1. torch.autograd through gfcc: G_pq(w) on 20 frequencies of the window for the p set, loss
       L = sum_w A(w)^2 + sum |G|^2, backward to w, eta and t2 (adjoint solves with the transposed sigma;
       the forward solutions are recomputed for the t2 gradient). Timed.
    2. Central finite differences, step 1e-5: dG/dw and dG/deta at all 20 frequencies (every p, q) from
       forward solves at w +- h and eta +- h against the adjoint-solve derivatives, and dL/dt2 along a
       random antisymmetric direction (two more contexts at t2 +- h dt2) against the autograd gradient.
    3. dG/dw-driven MOR: the derivative indicator on, 8 seeds, refined to 1e-6 on 500 points, evaluated
       on the workload's output grid (2000 points for adenine); its G points/s, and its A and G errors
       against the full solutions at the 20 frequencies of step 1."""
    import torch
    from paper_1902_06016_gb300 import Context, load
    from paper_1902_06016_gb300.autograd import green, spectral
    torch.cuda.set_device(0)
    load()
    W = synth.WORKLOADS[args.workload]
    o, v, eta0 = W["o"], W["v"], W["eta"]
    nw = args.nomega or W["nw"]
    t_gen = time.perf_counter()
    inp = synth.make_inputs(o, v, W["seed"])
    t_gen = time.perf_counter() - t_gen
    porb = list(range(o + v)) if args.pset == "all" else list(range(o))
    ws = np.linspace(W["wmin"], W["wmax"], 20)
    h = 1e-5
    stream = torch.cuda.current_stream()
    tol = 1e-10   # GMRES-IR reaches about 1e-11 with 41-bit exact-slice residuals; 1e-10 leaves a margin
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = Context(inp, tol=tol, precision=args.precision, stream=stream.cuda_stream, restart=args.restart)
    torch.cuda.synchronize()
    t_init = time.perf_counter() - t0
    if args.model_only:   # only the derivative-driven model, checked against full solves at 4 of the 20 frequencies
        ws = ws[::5]
        G_np = ctx.solve_full(ws, eta0, porb, want_A=False)["G"]
        A_np = -np.imag(np.einsum("wpp->w", G_np)) / np.pi
        out = {"metric": "G_pq(w) points/s, dG/dw-driven MOR + mixed precision", "value": None, "unit": UNIT,
               "n_gpus": 1, "mode": "autograd (model only)", "higher_is_better": True, "data": "synthetic",
               "dtype": f"c128 (f64 residuals, {args.precision} tensor-core inner sigma)",
               "config": {"workload": args.workload, "o": o, "v": v, "D": inp.dim, "n_p": len(porb), "eta": eta0,
                          "solve_tol": tol, "n_omega": nw, "max_batch": args.max_batch},
               "seconds": {"input_generation_host": t_gen, "gfcc_init": t_init}}

        def rel(a, b):
            return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))
    else:
        # 1. autograd forward + backward
        w_t = torch.tensor(ws, dtype=torch.float64, requires_grad=True)
        e_t = torch.tensor(eta0, dtype=torch.float64, requires_grad=True)
        t2_t = torch.tensor(inp.t2, dtype=torch.float64, requires_grad=True)
        t0 = time.perf_counter()
        G = green(w_t, e_t, ctx, porb, t2=t2_t)
        loss = (spectral(G) ** 2).sum() + (G.abs() ** 2).sum()
        loss.backward()
        torch.cuda.synchronize()
        t_ad = time.perf_counter() - t0
        G_np = G.detach().numpy()
        # 2. finite differences
        _, dw, de = ctx.green_derivatives(ws, eta0, porb)
        t0 = time.perf_counter()
        Gp = ctx.solve_full(ws + h, eta0, porb, want_A=False)["G"]
        Gm = ctx.solve_full(ws - h, eta0, porb, want_A=False)["G"]
        fd_w = (Gp - Gm) / (2 * h)
        Gp = ctx.solve_full(ws, eta0 + h, porb, want_A=False)["G"]
        Gm = ctx.solve_full(ws, eta0 - h, porb, want_A=False)["G"]
        fd_e = (Gp - Gm) / (2 * h)
        rng = np.random.default_rng(7)
        dt2 = rng.standard_normal(inp.t2.shape)
        dt2 = dt2 - dt2.transpose(1, 0, 2, 3)
        dt2 = dt2 - dt2.transpose(0, 1, 3, 2)
        dt2 *= np.abs(inp.t2).max() / np.abs(dt2).max()

        def loss_at(t2x):
            fields = {k: getattr(inp, k) for k in inp.__dataclass_fields__}
            fields["t2"] = t2x                     # lambda_2 held fixed at the original amplitudes
            cx = Context(synth.Inputs(**fields), tol=tol, precision=args.precision, stream=stream.cuda_stream,
                         restart=args.restart)
            Gx = cx.solve_full(ws, eta0, porb, want_A=False)["G"]
            cx.close()
            Ax = -np.imag(np.einsum("wpp->w", Gx)) / np.pi
            return float((Ax ** 2).sum() + (np.abs(Gx) ** 2).sum())

        fd_t2 = (loss_at(inp.t2 + h * dt2) - loss_at(inp.t2 - h * dt2)) / (2 * h)
        t_fd = time.perf_counter() - t0
        ad_t2 = float((t2_t.grad.numpy() * dt2).sum())
        # the scalar derivatives of the loss with respect to w_k and eta, from the finite differences of G
        A_np = -np.imag(np.einsum("wpp->w", G_np)) / np.pi

        def dloss(dG):
            dA = -np.imag(np.einsum("wpp->w", dG)) / np.pi
            return 2 * A_np * dA + 2 * np.real(np.conj(G_np) * dG).sum(axis=(1, 2))

        fd_loss_w = dloss(fd_w)
        fd_loss_e = float(dloss(fd_e).sum())

        def rel(a, b):
            return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))

        out = {"metric": "G_pq(w) points/s, dG/dw-driven MOR + mixed precision", "value": None,
               "unit": UNIT, "n_gpus": 1, "mode": "autograd", "higher_is_better": True, "data": "synthetic",
               "dtype": f"c128 (f64 residuals, {args.precision} tensor-core inner sigma, adjoint on the transposed sigma)",
               "config": {"workload": args.workload, "o": o, "v": v, "D": inp.dim, "n_p": len(porb), "eta": eta0,
                          "fd_omegas": 20, "fd_step": h, "solve_tol": tol, "n_omega": nw},
               "seconds": {"input_generation_host": t_gen, "gfcc_init": t_init,
                           "autograd_forward_backward": t_ad, "finite_differences": t_fd},
               "autograd_vs_fd": {
                   "dG_domega_rel_err": rel(dw, fd_w), "dG_deta_rel_err": rel(de, fd_e),
                   "dL_domega_rel_err": rel(w_t.grad.numpy(), fd_loss_w),
                   "dL_deta_rel_err": abs(float(e_t.grad) - fd_loss_e) / max(abs(fd_loss_e), 1e-300),
                   "dL_dt2_directional": {"autograd": ad_t2, "finite_difference": fd_t2,
                                          "rel_err": abs(ad_t2 - fd_t2) / max(abs(fd_t2), 1e-300)}}}
    print("autograd part: " + json.dumps(out), file=sys.stderr, flush=True)   # kept if the model step fails
    ctx.close()

    # 3. derivative-driven MOR on the output grid, in a fresh context (the adjoint operators, their
    # low-precision and exact-slice states and the gradient scratch of steps 1-2 are released first)
    from paper_1902_06016_gb300 import GfccError
    grid = np.linspace(W["wmin"], W["wmax"], nw)
    ctx = Context(inp, tol=args.solve_tol, precision=args.precision, stream=stream.cuda_stream, restart=args.restart,
                  deriv_indicator=True, max_batch=args.max_batch)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:
        e0.record(stream)
        ctx.mor_build(synth.omega_grid(W["wmin"], W["wmax"], args.seeds), eta0, porb)
        ref = ctx.mor_refine(W["wmin"], W["wmax"], args.ngrid, args.mor_tol, args.m_max)
        ev = ctx.mor_eval(grid)
        e1.record(stream)
        torch.cuda.synchronize()
        mor_ms = e0.elapsed_time(e1)
        at20 = ctx.mor_eval(ws)
        info = ctx.mor_info()
        out["value"] = nw * len(porb) / (mor_ms / 1e3)
        out["seconds"]["mor_ms"] = mor_ms
        out["mor"] = {"model_order": info["m"], "sampled_freqs": len(info["sampled"]), "converged": ref["converged"],
                      "max_err": ref["max_err"], "deriv_indicator": True,
                      "A_rel_err_vs_full_at_fd_omegas": rel(at20["A"], A_np),
                      "G_rel_err_vs_full_at_fd_omegas": rel(at20["G"], G_np),
                      "spectrum": spectrum_peaks(ev["A"], grid)}
    except GfccError as e:
        free_b, total_b = torch.cuda.mem_get_info()
        out["mor"] = {"error": str(e), "device_free_gb": free_b / 1e9, "device_total_gb": total_b / 1e9}
    ctx.close()
    return out


def oracle_sample(args, ncols, inp=None):
    """Time the FP64 CPU oracle on a bounded sample: full GMRES solves of ncols (w, p) points."""
    from oracle import bc, hbar
    from oracle import solve as sv
    W = synth.WORKLOADS[args.workload]
    if inp is None:
        inp = synth.make_inputs(W["o"], W["v"], W["seed"])
    hb = hbar.build(inp)
    porb = list(range(ncols))
    B = bc.b_vectors(inp, porb)
    w = [0.5 * (W["wmin"] + W["wmax"])]
    t0 = time.perf_counter()
    X, res = sv.gmres_solve(hb, B, w, W["eta"], tol=args.solve_tol)
    dt = time.perf_counter() - t0
    qset = orbital_set(args.workload, W["o"], W["o"] + W["v"])
    Gq = sv.green(bc.c_vectors(inp, qset), X)[0]     # [ncols, nq]: p = 0..ncols-1
    return {"value": ncols / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{ncols} full-dimension FP64 GMRES solve(s) (tol {args.solve_tol}) at w = {w[0]} Ha, "
                      f"p = 0..{ncols - 1}, {args.workload}; H-bar build and input generation untimed",
            "seconds": dt, "_G": Gq}


def ea_oracle_sample(args, ncols, inp):
    """The attachment oracle on a bounded sample: full GMRES solves (IP form, frequency -w) of the first
    ncols free terms of the p set at the middle of the attachment window."""
    from oracle import ea
    from oracle import solve as sv
    W = synth.WORKLOADS[args.workload]
    hb = ea.build(inp)
    porb = ea_orbital_set(args.workload, inp) if args.pset != "all" else list(range(inp.n))
    Bp, Cp = ea.ip_form(inp, hb, porb[:ncols], porb)
    w = [0.5 * sum(window(args, W))]
    t0 = time.perf_counter()
    Y, res = sv.gmres_solve(hb, Bp, [-w[0]], W["eta"], tol=args.solve_tol)
    dt = time.perf_counter() - t0
    Gq = sv.green(Cp, Y)[0]
    return {"value": ncols / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{ncols} full-dimension FP64 GMRES solve(s) of the attachment systems (tol {args.solve_tol}) "
                      f"at w = {w[0]} Ha, the first {ncols} orbital(s) of the p set, {args.workload}; H-bar build "
                      f"and input generation untimed", "seconds": dt, "_G": Gq}


def run_reference(args):
    """The oracle on the host cores, in bounded steps. Set-up (untimed): inputs, the oracle's H-bar
    build, and one full GMRES solve of (w_mid, p = 0) that gives the number of operator applications a
    G point costs. Each warm-up and timed step then runs ref_iters GMRES iterations of the same system
    (the oracle's own solver, capped), i.e. a known fraction of one G point; value = that fraction / the
    median step time, in G points per second."""
    from oracle import bc, hbar
    from oracle import sigma as sg
    from oracle import solve as sv
    W = synth.WORKLOADS[args.workload]
    inp = synth.make_inputs(W["o"], W["v"], W["seed"])
    hb = hbar.build(inp)
    b0 = bc.b_vectors(inp, [0])[0]
    w = 0.5 * (W["wmin"] + W["wmax"])
    diag = sg.diagonal(hb)
    calls = [0]

    def mv(x):
        calls[0] += 1
        return sg.sigma(hb, x)

    t0 = time.perf_counter()
    _, hist, ok = sv.gmres(mv, b0, w - 1j * W["eta"], diag, tol=args.solve_tol, restart=30, maxiter=3000)
    t_full = time.perf_counter() - t0
    n_full = calls[0]
    times, fracs = [], []
    for k in range(args.warmup + max(1, args.steps)):
        calls[0] = 0
        t0 = time.perf_counter()
        sv.gmres(mv, b0, w - 1j * W["eta"], diag, tol=args.solve_tol, restart=30, maxiter=args.ref_iters)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            fracs.append(calls[0] / n_full)
    t_med = statistics.median(times)
    v = statistics.median(fracs) / t_med
    cb = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
          "sample": f"{args.workload}, w = {w} Ha, p = 0: per step {args.ref_iters} GMRES iterations of the oracle "
                    f"({int(round(statistics.median(fracs) * n_full))} of the {n_full} operator applications of the "
                    f"full solve to tol {args.solve_tol}, which took {t_full:.1f} s untimed); inputs and H-bar build "
                    f"untimed", "full_solve_s": t_full, "full_solve_converged": bool(ok),
          "step_s_median": t_med}
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_med * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": args.workload, "o": W["o"], "v": W["v"], "D": inp.dim, "eta": W["eta"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if args.mode == "sigma":
        print(json.dumps(run_sigma(args)), flush=True)
        return
    if args.mode == "peaks":
        print(json.dumps(run_peaks(args)), flush=True)
        return
    if args.mode == "autograd":
        print(json.dumps(run_autograd(args)), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    inp, out = run_ours(args, rank, world)
    if rank == 0:
        full = out.get("full_fp64")
        if args.cpu_sample > 0 and args.sector == "ea" and inp.v > 130:
            out["cpu_baseline"] = {"skipped": "the attachment oracle holds full v^4 arrays; sampled up to v = 130"}
        elif args.cpu_sample > 0:
            try:
                cb = (ea_oracle_sample if args.sector == "ea" else oracle_sample)(args, args.cpu_sample, inp)
                Go = cb.pop("_G")
                if full is not None:   # the GPU results at the oracle's frequency, p = 0..ncols-1
                    k = Go.shape[0]
                    scale = np.abs(Go).max()
                    out["oracle_check"] = {
                        "points": int(Go.size), "omega": 0.5 * (synth.WORKLOADS[args.workload]["wmin"] +
                                                                synth.WORKLOADS[args.workload]["wmax"]),
                        "full_fp64_G_rel_err": None if args.siso else float(np.abs(full["_G_mid"][:k] - Go).max() / scale),
                        "mor_G_rel_err": float(np.abs(full["_G_mor_mid"][:k, 0] - Go[np.arange(k), np.arange(k)]).max()
                                               / scale) if args.siso else
                        float(np.abs(full["_G_mor_mid"][:k] - Go).max() / scale)}
                out["cpu_baseline"] = cb
            except Exception as e:  # the baseline must not hide the GPU line
                out["cpu_baseline"] = {"error": str(e)}
        if full is not None:
            full.pop("_G_mid", None)
            full.pop("_G_mor_mid", None)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
