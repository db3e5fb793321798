"""Benchmark of the ISCI sigma step sigma = H_tau c on GB300.

Workload (default): full CI, 2 alpha + 2 beta electrons in 60 orbitals
(1770^2 = 3,132,900 determinants), seeded synthetic integrals (decay length
4, 60 Cholesky vectors), screening threshold tau = 1e-14, FP64.  One step is
one sigma = H_tau c on a seeded unit vector resident in HBM.  The metric is
GUpdates/s, an update being one sigma_I += sign * unit * c_J over surviving
integral units and in-space determinant pairs (counted exactly at set-up).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload fci_n60] [--tau 1e-14] [--precision 64|32]
                  [--mixed-workload fci_n100|none] [--mixed-roots 3]

Beside the sigma line (rank 0, one GPU) it runs the precision form: FP32-mixed
and plain FP64 Davidson for the lowest roots of --mixed-workload, with the
energies' difference, iteration counts and the speedup ("mixed_precision").

Under torchrun (N > 1) every rank runs an independent replica of the
workload (the sigma step has no data-parallel exchange at one problem per
GPU); value = all ranks' updates / max over ranks of the timed span.
"""
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

METRIC = "σ-vector ms & GUpdates/s, HBM % of peak; FP32-mixed vs FP64 at |ΔE|≤1e-9 Eh"
FALLBACK_HBM_GBS = 6800.0
FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 rate (no FP64 figure in MEASURED_PEAKS.json)
BF16_FALLBACK_TFLOPS = 1900.0  # dense bf16, recipe fallback (burst) when MEASURED_PEAKS.json is absent
FP32_PEAK_TFLOPS = 80.5   # 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz
L2_FLUSH_BYTES = 512 << 20
ORACLE_UPDATES_PER_S = 2.0e8  # the row-wise oracle on 16 Grace cores (sizes its samples)

WORKLOADS = {
    "fci_n60": dict(n=60, na=2, nb=2, kmax=4, ell=4.0, nchol=60, box=False, seed=1000, tau=1e-14,
                    taus=(1e-14, 1e-12, 1e-10)),
    "fci_n10": dict(n=10, na=2, nb=2, kmax=4, ell=3.0, nchol=20, box=False, seed=0, tau=1e-14),
    "fci_n100": dict(n=100, na=2, nb=2, kmax=4, ell=5.0, nchol=20, box=False, seed=3000, tau=1e-12),
    "cisd_n200": dict(n=200, na=2, nb=2, kmax=2, ell=5.0, nchol=20, box=True, seed=2000, tau=1e-14),
    "cisdt_n100": dict(n=100, na=2, nb=2, kmax=3, ell=5.0, nchol=20, box=True, seed=2000, tau=1e-14),
    "cisd_n50": dict(n=50, na=2, nb=2, kmax=2, ell=5.0, nchol=20, box=True, seed=2000, tau=1e-14),
    "cisd_n100": dict(n=100, na=2, nb=2, kmax=2, ell=5.0, nchol=20, box=True, seed=2000, tau=1e-14),
    "cisd_n150": dict(n=150, na=2, nb=2, kmax=2, ell=5.0, nchol=20, box=True, seed=2000, tau=1e-14),
    "cisdt_n50": dict(n=50, na=2, nb=2, kmax=3, ell=5.0, nchol=20, box=True, seed=2000, tau=1e-14),
    "cisdt_n150": dict(n=150, na=2, nb=2, kmax=3, ell=5.0, nchol=20, box=True, seed=2000, tau=1e-14),
    "cisdt_n200": dict(n=200, na=2, nb=2, kmax=3, ell=5.0, nchol=20, box=True, seed=2000, tau=1e-14),
    # the batching form's block Davidson (16 roots, FP32-mixed)
    "cisdt_n120": dict(n=120, na=2, nb=2, kmax=3, ell=5.0, nchol=20, box=True, seed=4500, tau=1e-14),
    # more electrons per spin (strings of 3 and 4 electrons), full CI of about fci_n60's size
    "fci_n24_3a3b": dict(n=24, na=3, nb=3, kmax=6, ell=4.0, nchol=24, box=False, seed=5000, tau=1e-14),
    "fci_n16_4a4b": dict(n=16, na=4, nb=4, kmax=8, ell=4.0, nchol=16, box=False, seed=5100, tau=1e-14),
}


# the screening sweep: a workload whose integrals decay with the box, and thresholds
SCREEN_SWEEP = ("cisdt_n100", (1e-14, 1e-10, 1e-8, 1e-6, 1e-4))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (the job's time is
    its slowest rank's); the values themselves when there is one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(units_per_rank, ws, seconds):
    """Units all ranks processed per second: every rank does the same work (weak
    scaling), and the job takes as long as its slowest rank."""
    return ws * units_per_rank / seconds


def shard(count, rank, ws):
    """The instances of a many-instance workload that this rank runs: every
    ws-th one starting at rank, so ranks share the mix of sizes evenly and no
    instance is run twice or left out; instances are independent, so the
    shards need no exchange."""
    return list(range(rank, count, ws))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class NvmlClockSampler:
    """SM clock and clock-event (throttle) reasons read through NVML (the
    driver's libnvidia-ml, via ctypes) every ~2 ms in a thread during the timed
    region, so that even a region of tens of milliseconds gets many samples.
    Falls back to the nvidia-smi sampler when NVML cannot be loaded."""

    # NVML clock-event reason bits (nvml.h): software power cap, hardware
    # slowdown, software thermal slowdown, hardware thermal slowdown
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, index):
        import ctypes
        self.ct = ctypes
        self.fallback = None
        self.samples, self.reasons, self.smax = [], set(), None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) != 0:
                raise OSError("no NVML device %d" % index)
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx)) == 0:
                self.smax = float(mx.value)
            self.lib, self.h = lib, h
            fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
            self.reason_fn = fn or lib.nvmlDeviceGetCurrentClocksThrottleReasons
        except (OSError, AttributeError):
            self.fallback = ClockSampler(index)

    def _poll(self):
        ct = self.ct
        mhz, rs = ct.c_uint(), ct.c_ulonglong()
        while not self.stop_flag:
            if self.lib.nvmlDeviceGetClockInfo(self.h, ct.c_int(1), ct.byref(mhz)) == 0:
                self.samples.append(float(mhz.value))
            if self.reason_fn(self.h, ct.byref(rs)) == 0:
                for nm, bit in self.BITS.items():
                    if rs.value & bit:
                        self.reasons.add(nm)
            time.sleep(0.002)

    def start(self):
        if self.fallback:
            return self.fallback.start()
        self.stop_flag = False
        self.thread = threading.Thread(target=self._poll, daemon=True)
        self.thread.start()

    def stop(self):
        if self.fallback:
            return self.fallback.stop()
        self.stop_flag = True
        self.thread.join(timeout=5)
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None, "sm_max_mhz": self.smax,
                "reasons": sorted(self.reasons), "samples": len(self.samples), "source": "nvml"}


def _peaks_file():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            pass
    return None


def measured_peaks():
    d = _peaks_file()
    if d:
        for key in ("hbm_gbs", "hbm_GBs", "hbm"):
            if key in d:
                return float(d[key]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def bf16_peak():
    d = _peaks_file()
    if d and "bf16_tflops" in d:
        return float(d["bf16_tflops"]), "measured (burst)"
    return BF16_FALLBACK_TFLOPS, "fallback (burst)"


def profile_traffic(kernel_key):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary,
    or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        d = json.load(f)
    ent = d.get(kernel_key)
    if not ent:
        return None, None
    # every source the launch depends on (the kernel, and the code that builds
    # its work list) must be unchanged since the capture
    for src_rel, want in ent.get("sources", {ent.get("source"): ent.get("source_sha256_16")}).items():
        src = os.path.join(ROOT, src_rel or "")
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] if src_rel and os.path.exists(src) else None
        if h != want:
            return None, ent
    return float(ent["dram_bytes_per_launch"]), ent


def run_ours(args, wl, ws, rank, local):
    import numpy as np
    import torch

    from paper_1609_07757_gb300 import _lib as L
    from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tau = args.tau if args.tau is not None else wl["tau"]
    h1, eri = make_integrals(wl["n"], wl["seed"], ell=wl["ell"], nchol=wl["nchol"], box=wl["box"])
    stream = torch.cuda.current_stream()
    L.iscsi_set_stream(stream)
    L.iscsi_set_option("autotune", args.autotune)
    t0 = time.time()
    L.iscsi_init(wl["n"], wl["na"], wl["nb"], wl["kmax"], h1, eri, tau)
    init_s = time.time() - t0
    ndet = L.iscsi_ndet()
    updates = L.iscsi_updates_per_sigma()
    c = torch.tensor(unit_vector(ndet, 17 + rank), dtype=torch.float64, device=dev)
    s = torch.empty_like(c)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    L.iscsi_set_option("precision", args.precision)

    for _ in range(args.warmup):
        L.iscsi_sigma(c, s, 1)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # device-timed region: K sigma steps, L2 flushed between them
    L.iscsi_set_option("phase_timing", 1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = NvmlClockSampler(local)
    clocks.start()
    barrier()
    wall0 = time.time()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        L.iscsi_sigma(c, s, 1)
        ev[k][1].record(stream)
    barrier()
    wall = time.time() - wall0
    clk = clocks.stop()
    st = L.iscsi_stats()
    L.iscsi_set_option("phase_timing", 0)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)

    # end-to-end through the host-buffer C-ABI call (pinned buffers, copies timed)
    ch = torch.empty(ndet, dtype=torch.float64, pin_memory=True)
    ch.copy_(c.cpu())
    sh = torch.empty(ndet, dtype=torch.float64, pin_memory=True)
    ch_np, sh_np = ch.numpy(), sh.numpy()
    L.iscsi_sigma_host(ch_np, sh_np, 1)
    barrier()
    e0 = time.time()
    for _ in range(args.steps):
        L.iscsi_sigma_host(ch_np, sh_np, 1)
    barrier()
    e2e_s = time.time() - e0
    ref = s.cpu().numpy()
    e2e_ok = bool(np.array_equal(sh_np, ref))

    tot_ms, e2e_s = max_over_ranks([tot_ms, e2e_s], device=dev)
    ms = tot_ms / args.steps
    value = whole_job_rate(updates, ws, ms * 1e-3) / 1e9
    e2e_val = whole_job_rate(updates * args.steps, ws, e2e_s) / 1e9

    # roofline of the dominant kernel (opposite-spin contraction)
    gemm_ms = st["phase_ms"]["opposite_gemm"] / max(1, st["timed_calls"])
    tc = st.get("fp64_tc" if args.precision == 64 else "fp32_tc", 0) == 1
    route = st.get("route_fp%d" % args.precision, {})
    tc = tc and route.get("ab_tc", 1) == 1
    # with both contractions on the tensor cores they are one launch: its flops
    # are the opposite- and the same-spin slice products
    both = st.get("both_tc_fp%d" % args.precision, 0) == 1
    what = "opposite- and same-spin contractions in one launch" if both else "opposite-spin contraction"
    tag = "_both" if both else ""
    if tc and args.precision == 64:
        # tensor-core kernel: bf16 MMA flops its schedule issues (the exact slice
        # products of live slices of non-screened blocks, over whole tiles)
        flops = st.get("tc_schedule_fp64", {}).get("issued_bf16_flops") or (
            st["opposite_tc_bf16_flops"] + (st.get("samespin_tc_bf16_flops", 0.0) if both else 0.0))
        peak, peak_src = bf16_peak()
        bound, kname, kkey = "tensor", "k_oz_gemm (tcgen05, FP64-accurate %s)" % what, \
            "k_oz_gemm%s_%s" % (tag, args.workload)
    elif tc:
        # FP32 form: 6 of the 9 products of three bf16 terms per operand
        flops = (st["opposite_tc_bf16_flops"] + (st.get("samespin_tc_bf16_flops", 0.0) if both else 0.0)) * 6.0 / 28.0
        peak, peak_src = bf16_peak()
        bound, kname, kkey = "tensor", "k_tc32w_gemm (tcgen05, FP32-accurate %s, 128 x 128 tiles)" % what, \
            "k_tc32w_gemm%s_%s" % (tag, args.workload)
    else:
        flops = st["opposite_gemm_flops"]
        peak = FP64_PEAK_TFLOPS if args.precision == 64 else FP32_PEAK_TFLOPS
        peak_src = ("FP64 rate of GB300 (1.25 TFLOP/s; own probe measured 1.198)" if args.precision == 64
                    else "152 SM x 128 FFMA/clk x 2.07 GHz")
        bound, kname = "alu", "k_grouped_gemm (opposite-spin contraction)"
        kkey = "k_grouped_gemm_fp%d_%s" % (args.precision, args.workload)
    achieved = flops / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else None
    traffic, _ = profile_traffic(kkey)
    hbm_peak, hbm_src = measured_peaks()
    esz = 8 if args.precision == 64 else 4
    npairs = wl["n"] ** 2
    # compulsory bytes of one sigma: c read, sigma written, the surviving opposite-spin
    # units and the same-spin string Hamiltonians read once
    nstr = st["nstrings"][0]
    comp_bytes = esz * (2 * ndet + npairs * npairs + 2 * nstr * nstr)
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "GUpdates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f64 (tcgen05 bf16 exact slices, int64/f64 accumulation)" if tc else "f64")
        if args.precision == 64 else ("f32 (tcgen05, three bf16 terms, f32 accumulation)" if tc else "f32"),
        "data": "synthetic (seeded integrals shaped like the paper's Be-in-a-box sets)",
        "config": {"workload": args.workload, "norb": wl["n"], "nalpha": wl["na"], "nbeta": wl["nb"],
                   "max_excitation": wl["kmax"], "ndet": ndet, "tau": tau, "nvec": 1,
                   "updates_per_sigma": updates, "l2": "flushed between steps (512 MiB write)",
                   "parallelism": "replicas" if ws > 1 else "single-gpu"},
        "gpu_launches": None,
        "e2e": {"value": round(e2e_val, 3), "unit": "GUpdates/s", "h2d_bytes_per_step": 8 * ndet,
                "d2h_bytes_per_step": 8 * ndet, "matches_device_path": e2e_ok},
        "roofline": {"bound": bound, "achieved": round(achieved, 4) if achieved else None, "peak": peak,
                     "unit": "TFLOP/s", "frac": round(achieved / peak, 4) if achieved else None,
                     "traffic": traffic, "kernel": kname, "kernel_ms": round(gemm_ms, 4), "flops_per_launch": flops,
                     "fp64_equivalent_tflops": round(st["opposite_gemm_flops"] / (gemm_ms * 1e-3) / 1e12, 3)
                     if gemm_ms > 0 else None,
                     # the method's own work: one multiply-add (2 flops) per surviving update
                     "method_flops_per_launch": 2.0 * updates,
                     "method_tflops": round(2.0 * updates / (gemm_ms * 1e-3) / 1e12, 3) if gemm_ms > 0 else None,
                     "method_frac": round(2.0 * updates / (gemm_ms * 1e-3) / 1e12 / peak, 5) if gemm_ms > 0 else None,
                     "emulation_factor": round(flops / (2.0 * updates), 3) if updates > 0 else None,
                     "schedule": st.get("tc_schedule_fp64") if (tc and args.precision == 64) else None,
                     "peak_source": peak_src},
        "hbm": {"compulsory_bytes_per_step": comp_bytes,
                "achieved_gbs": round(comp_bytes / (ms * 1e-3) / 1e9, 2),
                "peak_gbs": hbm_peak, "frac": round(comp_bytes / (ms * 1e-3) / 1e9 / hbm_peak, 5),
                "peak_source": hbm_src},
        "phase_ms_per_step": {k: round(v / max(1, st["timed_calls"]), 4) for k, v in st["phase_ms"].items()},
        "clocks": clk,
        "wall_s_timed": round(wall, 3),
        "init_s": round(init_s, 3),
    }
    # kernel launches of the library inside the timed region (counted by the library)
    line["gpu_launches"] = st.get("kernel_launches")
    line["config"]["opposite_units_kept"] = round(st["units_kept_opposite"] / max(1, st["units_total"]["opposite"]), 6)
    if ws == 1 and args.roots > 0:
        # the lowest roots of the same context, pinned to the oracle
        line["roots"] = run_roots(L, wl, tau, args.roots, with_oracle=not args.no_cpu_baseline,
                                  full_oracle=args.oracle_full)
    L.iscsi_finalize()
    if ws == 1 and args.tau_sweep:
        # the same sigma at the workload's other screening thresholds
        line["tau_sweep"] = run_tau_sweep(L, wl, [t for t in wl.get("taus", ()) if t != tau], steps=args.steps,
                                          warmup=args.warmup)
        # where the screen removes whole blocks of units: the box-decay CISDT
        # workload at rising thresholds (sigma time against the units kept)
        sw = WORKLOADS[SCREEN_SWEEP[0]]
        line["screen_sweep"] = {"workload": SCREEN_SWEEP[0],
                                "points": run_tau_sweep(L, sw, SCREEN_SWEEP[1], steps=args.steps, warmup=args.warmup)}
    return line


def run_tau_sweep(L, wl, taus, steps=5, warmup=3):
    """sigma time, survivor fraction, updates and the contraction's time at other
    screening thresholds tau (L2 flushed between steps)."""
    import torch

    from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

    h1, eri = make_integrals(wl["n"], wl["seed"], ell=wl["ell"], nchol=wl["nchol"], box=wl["box"])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = []
    for tau in taus:
        L.iscsi_init(wl["n"], wl["na"], wl["nb"], wl["kmax"], h1, eri, tau)
        nd = L.iscsi_ndet()
        c = torch.tensor(unit_vector(nd, 17), dtype=torch.float64, device="cuda")
        s = torch.empty_like(c)
        for _ in range(warmup):
            L.iscsi_sigma(c, s, 1)
        L.iscsi_set_option("phase_timing", 1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record()
            L.iscsi_sigma(c, s, 1)
            ev[k][1].record()
        torch.cuda.synchronize()
        st = L.iscsi_stats()
        L.iscsi_set_option("phase_timing", 0)
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        upd = L.iscsi_updates_per_sigma()
        sched = st.get("tc_schedule_fp64", {})
        out.append({"tau": tau, "sigma_ms": round(ms, 4), "gupdates_per_s": round(upd / (ms * 1e-3) / 1e9, 1),
                    "updates_per_sigma": upd,
                    "opposite_units_kept": round(st["units_kept_opposite"] / max(1, st["units_total"]["opposite"]), 6),
                    "contraction_ms": round(st["phase_ms"]["opposite_gemm"] / max(1, st["timed_calls"]), 4),
                    "issued_bf16_flops": sched.get("issued_bf16_flops")})
        L.iscsi_finalize()
    return out


def oracle_pin_roots(o, energies, x, w, sample_rows, seed=23):
    """Pin approximate eigenpairs (E, x) of the GPU (w = H x by the GPU) to the
    oracle on sampled rows I: the oracle's (H x)_I against the GPU's, and the
    residual estimate ||r||^2 ~ ndet / m sum_I (r_I)^2 with r = H_oracle x - E x.
    With the gap delta of each root to its computed neighbours, the a-posteriori
    bound |E - lambda| <= ||r||^2 / delta (Kato-Temple, for the Rayleigh
    quotient) is reported from the GPU's full residual and from the estimate."""
    import numpy as np

    nd = x.shape[1]
    rows = np.random.default_rng(seed).choice(nd, size=min(nd, sample_rows), replace=False)
    out = []
    for i, e in enumerate(energies):
        xi = x[i] / np.linalg.norm(x[i])
        wi = w[i] / np.linalg.norm(x[i])
        rho = float(xi @ wi)
        r_gpu = float(np.linalg.norm(wi - e * xi))
        so = o.sigma_rows(xi, rows)
        d = np.abs(so - wi[rows]).max()
        r_est = float(np.sqrt(nd / rows.size * np.sum((so - e * xi[rows]) ** 2)))
        gaps = [abs(e - f) for j, f in enumerate(energies) if j != i]
        gap = min(gaps) if gaps else None
        out.append({"energy": float(e), "rayleigh_gpu": rho, "abs_E_minus_rayleigh": abs(float(e) - rho),
                    "residual_gpu": r_gpu, "residual_oracle_estimate": r_est,
                    "oracle_vs_gpu_sigma_max_abs": float(d), "sigma_inf": float(np.abs(wi).max()),
                    "gap": gap, "bound_gpu": r_gpu ** 2 / gap if gap else None,
                    "bound_oracle_estimate": r_est ** 2 / gap if gap else None})
    return {"sample_rows": int(rows.size), "roots": out}


def run_roots(L, wl, tau, nroots=2, tol=1e-8, with_oracle=True, full_oracle=False, oracle_s=12.0):
    """The lowest `nroots` roots of the current context (device Davidson, FP64; one
    more root is computed for the gaps), each pinned to the oracle on a sample of
    rows sized for about oracle_s seconds of the oracle's work (or all rows with
    full_oracle, minutes at full CI in 60 orbitals)."""
    import numpy as np
    import torch

    import oracle
    from paper_1609_07757_gb300.synthetic import make_integrals

    nd = L.iscsi_ndet()
    k = nroots + 1
    vecs = torch.zeros((k, nd), dtype=torch.float64, device="cuda")
    L.iscsi_set_option("precision", 64)
    t0 = time.time()
    st, e = L.iscsi_davidson(k, tol, vecs)
    wall = time.time() - t0
    stt = L.iscsi_stats()
    w = torch.empty_like(vecs)
    L.iscsi_sigma(vecs, w, k)
    torch.cuda.synchronize()
    out = {"nroots": nroots, "tol": tol, "status": int(st), "energies": [float(x) for x in e[:nroots]],
           "next_energy": float(e[nroots]), "iterations": stt["davidson_iters"], "seconds": round(wall, 3)}
    if with_oracle:
        h1, eri = make_integrals(wl["n"], wl["seed"], ell=wl["ell"], nchol=wl["nchol"], box=wl["box"])
        o = oracle.Oracle(wl["n"], wl["na"], wl["nb"], wl["kmax"], tau, h1, eri)
        upd_row = L.iscsi_updates_per_sigma() / max(1, nd)
        rows = nd if full_oracle else int(oracle_s * ORACLE_UPDATES_PER_S / upd_row / nroots)
        t1 = time.time()
        pin = oracle_pin_roots(o, [float(x) for x in e], vecs.cpu().numpy(), w.cpu().numpy(), rows)
        pin["roots"] = pin["roots"][:nroots]
        pin["oracle_seconds"] = round(time.time() - t1, 2)
        pin["cores"] = len(os.sched_getaffinity(0))
        out["oracle_pin"] = pin
    return out


def run_precision_form(name, nroots=3, tol=1e-8, with_oracle=True, oracle_s=12.0):
    """FP32-mixed against plain FP64 Davidson on one workload: lowest roots, time,
    iterations (FP32 phase), and |dE| between the two.  Before the timed runs,
    untimed sigma calls with the vector counts the solvers use (1 and nroots:
    the block, and the FP64 re-evaluation after the FP32 phase, which runs in
    blocks of nroots) do the one-time operand preparation and routing trials,
    so that neither arm times them."""
    import numpy as np
    import torch

    from paper_1609_07757_gb300 import _lib as L
    from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

    wl = WORKLOADS[name]
    h1, eri = make_integrals(wl["n"], wl["seed"], ell=wl["ell"], nchol=wl["nchol"], box=wl["box"])
    L.iscsi_init(wl["n"], wl["na"], wl["nb"], wl["kmax"], h1, eri, wl["tau"])
    ndet = L.iscsi_ndet()
    c = torch.tensor(unit_vector(ndet, 5), dtype=torch.float64, device="cuda")
    s = torch.empty_like(c)
    out = {"workload": name, "ndet": ndet, "nroots": nroots, "tol": tol}
    res = {}
    orc = None
    cw = torch.tensor(np.stack([unit_vector(ndet, 5 + i) for i in range(nroots)]), dtype=torch.float64,
                      device="cuda")
    sw = torch.empty_like(cw)
    for prec, counts in ((64, (1, nroots)), (32, (1, nroots))):
        L.iscsi_set_option("precision", prec)
        for nv in counts:
            L.iscsi_sigma(cw, sw, nv)
    torch.cuda.synchronize()
    del cw, sw
    for prec in (64, 32):
        L.iscsi_set_option("precision", prec)
        L.iscsi_sigma(c, s, 1)
        torch.cuda.synchronize()
        vecs = torch.zeros((nroots, ndet), dtype=torch.float64, device="cuda")
        t0 = time.time()
        st, e = L.iscsi_davidson(nroots, tol, vecs)
        wall = time.time() - t0
        stt = L.iscsi_stats()
        # FP64 residual of the returned vectors (one FP64 sigma)
        L.iscsi_set_option("precision", 64)
        w = torch.empty_like(vecs)
        L.iscsi_sigma(vecs, w, nroots)
        torch.cuda.synchronize()
        et = torch.tensor(np.asarray(e), dtype=torch.float64, device="cuda")[:, None]
        rnorm = torch.linalg.norm(w - et * vecs, dim=1).cpu().numpy()
        res[prec] = {"status": int(st), "energies": [float(x) for x in e], "iters": stt["davidson_iters"],
                     "fp32_iters": stt.get("davidson_fp32_iters", 0), "ms": round(stt["davidson_ms"], 3),
                     "wall_s": round(wall, 3), "residual_norms": [float("%.3e" % r) for r in rnorm]}
        if with_oracle:
            # the returned eigenpairs pinned to the oracle on a sample of rows
            import oracle
            if orc is None:
                orc = oracle.Oracle(wl["n"], wl["na"], wl["nb"], wl["kmax"], wl["tau"], h1, eri)
            upd_row = L.iscsi_updates_per_sigma() / max(1, ndet)
            rows = int(oracle_s * ORACLE_UPDATES_PER_S / upd_row / (2 * nroots))
            t1 = time.time()
            pin = oracle_pin_roots(orc, [float(x) for x in e], vecs.cpu().numpy(), w.cpu().numpy(), rows)
            pin["oracle_seconds"] = round(time.time() - t1, 2)
            pin["cores"] = len(os.sched_getaffinity(0))
            res[prec]["oracle_pin"] = pin
    L.iscsi_set_option("precision", 64)
    L.iscsi_finalize()
    de = max(abs(a - b) for a, b in zip(res[32]["energies"], res[64]["energies"]))
    out.update({"fp64": res[64], "mixed": res[32], "max_abs_dE_mixed_vs_fp64": float("%.3e" % de),
                "within_1e-9": de <= 1e-9,
                "speedup_mixed_vs_fp64": round(res[64]["ms"] / res[32]["ms"], 3) if res[32]["ms"] > 0 else None})
    return out


def run_batching(count=64, reps=5, tau=1e-14, nroots=1, rank=0, ws=1):
    """The batching form: `count` independent full-CI instances (2 alpha + 2 beta
    electrons, orbital counts uniform on [20, 80], each with its own seeded
    integrals of the 10-orbital workload's generator).  sigma for all of them
    one context at a time (one iscsi_sigma per instance) against one
    iscsi_batch_sigma call (merged contractions, replayed CUDA graph), FP64 and
    FP32; then the lowest root of every instance by Davidson, one at a time."""
    import torch

    from paper_1609_07757_gb300 import _lib as L
    from paper_1609_07757_gb300.synthetic import make_integrals, multi_instance_sizes, unit_vector

    all_sizes = [int(x) for x in multi_instance_sizes(count)]
    mine = shard(count, rank, ws)  # with several ranks each runs its own share of the instances
    sizes = [all_sizes[i] for i in mine]
    hs, cs, ss, upd, ndets = [], [], [], 0.0, 0
    t0 = time.time()
    for i, n in zip(mine, sizes):
        h1, eri = make_integrals(n, 4000 + i, ell=3.0, nchol=20)
        L.iscsi_init(n, 2, 2, 4, h1, eri, tau)
        hs.append(L.iscsi_ctx_current())
        nd = L.iscsi_ndet()
        ndets += nd
        upd += L.iscsi_updates_per_sigma()
        c = torch.tensor(unit_vector(nd, 7 + i), dtype=torch.float64, device="cuda")
        cs.append(c)
        ss.append(torch.empty_like(c))
    init_s = time.time() - t0
    out = {"instances": count, "ranks": ws, "orbitals": [min(all_sizes), max(all_sizes)],
           "mean_ndet_rank0": ndets / max(1, len(mine)), "updates_per_round_rank0": upd, "init_s": round(init_s, 2)}
    for prec in (64, 32):
        L.iscsi_set_option("precision", prec)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def single():
            for h, c, s in zip(hs, cs, ss):
                L.iscsi_ctx_use(h)
                L.iscsi_sigma(c, s, 1)

        def batched():
            L.iscsi_batch_sigma(hs, cs, ss, 1)

        res = {}
        for name, fn in (("one_at_a_time", single), ("batched", batched)):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            w0 = time.time()
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            wall = (time.time() - w0) / reps
            ms = e0.elapsed_time(e1) / reps
            ms, wall = max_over_ranks([ms, wall], device="cuda")
            res[name] = {"ms_per_round": round(ms, 3), "host_wall_ms_per_round": round(wall * 1e3, 3),
                         "instances_per_s": round(count / (ms * 1e-3), 1),
                         "sigma_per_s": round(count / (ms * 1e-3), 1),
                         "GUpdates_per_s_rank0": round(upd / (ms * 1e-3) / 1e9, 1)}
        res["speedup"] = round(res["one_at_a_time"]["ms_per_round"] / res["batched"]["ms_per_round"], 3)
        out["fp%d" % prec] = res
    L.iscsi_set_option("precision", 64)
    # the lowest root of every instance: one Davidson per instance, then all
    # instances iterated together (iscsi_batch_davidson), FP64 and FP32-mixed
    import numpy as np
    for prec in (64, 32):
        L.iscsi_set_option("precision", prec)
        t0 = time.time()
        iters, e_single = 0, []
        for h in hs:
            L.iscsi_ctx_use(h)
            st, e = L.iscsi_davidson(nroots, 1e-8)
            e_single.append(e)
            iters += L.iscsi_stats()["davidson_iters"]
        torch.cuda.synchronize()
        dt1 = time.time() - t0
        t0 = time.time()
        st, e_batch, sts = L.iscsi_batch_davidson(hs, nroots, 1e-8)
        torch.cuda.synchronize()
        dt2 = time.time() - t0
        dt1, dt2 = max_over_ranks([dt1, dt2], device="cuda")
        de = float(np.abs(np.asarray(e_single) - e_batch).max())
        out["davidson_fp%d" % prec] = {
            "roots_per_instance": nroots, "one_at_a_time_s": round(dt1, 2), "batched_s": round(dt2, 2),
            "instances_per_s_one_at_a_time": round(count / dt1, 2), "instances_per_s_batched": round(count / dt2, 2),
            "speedup": round(dt1 / dt2, 3), "iterations_one_at_a_time": iters, "batched_status": st,
            "converged": int(sum(1 for x in sts if x == 0)), "max_abs_dE_batched_vs_single": float("%.3e" % de)}
    L.iscsi_set_option("precision", 64)
    L.iscsi_finalize()
    return out


def run_density(name, steps=10, warmup=3, with_cpu=True, tau=None):
    """One- and two-body density matrices (Eqs. d1, d2) of a unit vector on a
    workload: device ms per call (L2 flushed between calls), the contraction's
    launch time and tensor-core rate, and the oracle's element-wise route on a
    bounded sample of elements, scaled to the whole tensor."""
    import numpy as np
    import torch

    from paper_1609_07757_gb300 import _lib as L
    from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

    wl = WORKLOADS[name]
    tau = wl["tau"] if tau is None else tau
    h1, eri = make_integrals(wl["n"], wl["seed"], ell=wl["ell"], nchol=wl["nchol"], box=wl["box"])
    stream = torch.cuda.current_stream()
    L.iscsi_set_stream(stream)
    L.iscsi_init(wl["n"], wl["na"], wl["nb"], wl["kmax"], h1, eri, tau)
    n, ndet = wl["n"], L.iscsi_ndet()
    c = torch.tensor(unit_vector(ndet, 23), dtype=torch.float64, device="cuda")
    d1 = torch.empty((2, n, n), dtype=torch.float64, device="cuda")
    d2 = torch.empty((3, n, n, n, n), dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(max(3, warmup)):
        L.iscsi_density(c, None, d1, d2)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    gemm = []
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        L.iscsi_density(c, None, d1, d2)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    # the contraction's own launch time, read after further untimed calls
    for _ in range(3):
        flush.zero_()
        L.iscsi_density(c, None, d1, d2)
        gemm.append(L.iscsi_stats()["density_gemm_ms"])
    st = L.iscsi_stats()
    bf16, fp64 = st["density_bf16_flops"][0], st["density_fp64_flops"][0]
    gemm_ms = float(np.mean(gemm))
    peak, peak_src = bf16_peak()
    # invariants of a unit vector: traces of the blocks
    na, nb = wl["na"], wl["nb"]
    tr = [float(torch.einsum("pprr->", d2[b])) for b in range(3)]
    checks = {"trace_aa": tr[0], "trace_ab": tr[1], "trace_bb": tr[2],
              "expected": [na * (na - 1), na * nb, nb * (nb - 1)],
              "max_trace_err": max(abs(tr[0] - na * (na - 1)), abs(tr[1] - na * nb), abs(tr[2] - nb * (nb - 1)))}
    out = {"workload": name, "ndet": ndet, "ms_per_call": round(ms, 4), "contraction_ms": round(gemm_ms, 4),
           "contraction_bf16_flops": bf16, "contraction_fp64_flops": fp64,
           "roofline": {"bound": "tensor", "achieved": round(bf16 / (gemm_ms * 1e-3) / 1e12, 4), "peak": peak,
                        "unit": "TFLOP/s", "frac": round(bf16 / (gemm_ms * 1e-3) / 1e12 / peak, 4),
                        "traffic": profile_traffic("k_oz_gemm_density_%s" % name)[0],
                        "kernel": "k_oz_gemm<1> (tcgen05, FP64-accurate Gram products of lifted vectors, ket = bra)",
                        "peak_source": peak_src},
           "fp64_equivalent_tflops": round(fp64 / (gemm_ms * 1e-3) / 1e12, 3),
           "output_bytes": 8 * (2 * n * n + 3 * n ** 4), "l2": "flushed between calls", "checks": checks}
    L.iscsi_finalize()
    if with_cpu:
        # the oracle's element-wise route (every element a pass over all determinants)
        # on a sample of elements, scaled to the 3 n^4 + 2 n^2 elements
        from oracle import Oracle, max_threads
        o = Oracle(wl["n"], na, nb, wl["kmax"], tau, h1, eri)
        cc = unit_vector(ndet, 23)
        rng = np.random.default_rng(1)
        m = 2 * max_threads()
        for _ in range(2):  # calibrate on a few elements, then aim at ~10 s
            spec = np.column_stack([rng.integers(0, 3, m)] + [rng.integers(0, n, m) for _ in range(4)])
            t0 = time.time()
            vals = o.density_elems(cc, None, spec)
            dt = time.time() - t0
            if dt >= 3.0:
                break
            m = int(min(3 * n ** 4, max(m, m * 10.0 / max(dt, 1e-3))))
        full_s = dt / m * (3 * n ** 4 + 2 * n * n)
        out["cpu_baseline"] = {"value": round(full_s * 1e3, 1), "unit": "ms per density call (extrapolated)",
                               "cores": max_threads(), "kind": "oracle",
                               "sample": "%d random d2 elements by the oracle's element-wise route (%.1f s), "
                                         "scaled to all %d elements" % (m, dt, 3 * n ** 4 + 2 * n * n)}
        out["sample_check"] = {"elements": m, "max_abs_diff": float(np.abs(
            d2.cpu().numpy()[spec[:, 0], spec[:, 1], spec[:, 2], spec[:, 3], spec[:, 4]] - vals).max())}
    return out


def dipole_like(n):
    """A position-like one-body coupling (orbitals on a line), for the propagation leg."""
    import numpy as np
    v = np.diag(np.arange(n) - (n - 1) / 2.0) / n
    return v + 0.05 * (np.eye(n, k=1) + np.eye(n, k=-1))


def run_operators(name, electron_workloads=("fci_n24_3a3b", "fci_n16_4a4b"), steps=5, warmup=3):
    """Operators other than the Hamiltonian through the same sigma (Sec. "Second
    part": only the integrals change), on full CI: a transition operator
    a+_p a_q (one-body, not symmetric), a one-body operator D (dipole-like) and
    the two-body property operator D^2 (h1 = d d, (pq|rs) = 2 d_pq d_rs).  Each
    is timed (L2 flushed between calls) and checked by a closed form of its
    own: <x|A c> = <A^T x|c> for the transition operator, D^2 c = D (D c) for
    the square.  Then sigma of the Hamiltonian with 3 and 4 electrons per spin."""
    import numpy as np
    import torch

    from paper_1609_07757_gb300 import _lib as L
    from paper_1609_07757_gb300.synthetic import (make_integrals, square_operator_integrals, transition_operator,
                                                  unit_vector)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(c, s):
        for _ in range(warmup):
            L.iscsi_sigma(c, s, 1)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record()
            L.iscsi_sigma(c, s, 1)
            ev[k][1].record()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    def apply(c):
        s = torch.empty_like(c)
        L.iscsi_sigma(c, s, 1)
        return s

    wl = WORKLOADS[name]
    n, na, nb = wl["n"], wl["na"], wl["nb"]
    kfull = na + nb
    d = dipole_like(n)
    h2, eri2 = square_operator_integrals(d)
    p, q = n - 1, 0
    ops = {}
    handles = {}
    for key, h1, eri in (("transition", transition_operator(n, p, q), None),
                         ("transition_adjoint", transition_operator(n, q, p), None),
                         ("dipole", d, None), ("dipole_squared", h2, eri2)):
        L.iscsi_init(n, na, nb, kfull, h1, eri, 0.0)
        handles[key] = L.iscsi_ctx_current()
    nd = L.iscsi_ndet()
    c = torch.tensor(unit_vector(nd, 41), dtype=torch.float64, device="cuda")
    x = torch.tensor(unit_vector(nd, 42), dtype=torch.float64, device="cuda")
    for key in ("transition", "dipole", "dipole_squared"):
        L.iscsi_ctx_use(handles[key])
        s = torch.empty_like(c)
        ms = timed(c, s)
        upd = L.iscsi_updates_per_sigma()
        ops[key] = {"ms_per_sigma": round(ms, 4), "updates_per_sigma": upd,
                    "gupdates_per_s": round(upd / (ms * 1e-3) / 1e9, 1)}
    L.iscsi_ctx_use(handles["transition"])
    ac = apply(c)
    L.iscsi_ctx_use(handles["transition_adjoint"])
    atx = apply(x)
    lhs, rhs = float(torch.dot(x, ac)), float(torch.dot(atx, c))
    ops["transition"].update({"p": p, "q": q, "adjoint_check": {"x_Ac": lhs, "ATx_c": rhs,
                                                                "abs_diff": abs(lhs - rhs)}})
    L.iscsi_ctx_use(handles["dipole_squared"])
    s2 = apply(c)
    L.iscsi_ctx_use(handles["dipole"])
    dd = apply(apply(c))
    ops["dipole_squared"]["check_vs_d_twice"] = {
        "max_abs_diff_rel": float((s2 - dd).abs().max() / dd.abs().max())}
    L.iscsi_finalize()
    out = {"workload": name, "ndet": nd, "tau": 0.0, "operators": ops,
           "meaning": "transition: a+_%d a_%d (both spins); dipole: d = diag(p - (n-1)/2)/n + 0.05 "
                      "nearest-neighbour coupling; dipole_squared: D^2 as a two-body operator" % (p, q)}
    electrons = []
    for ename in electron_workloads:
        ew = WORKLOADS[ename]
        h1, eri = make_integrals(ew["n"], ew["seed"], ell=ew["ell"], nchol=ew["nchol"], box=ew["box"])
        L.iscsi_init(ew["n"], ew["na"], ew["nb"], ew["kmax"], h1, eri, ew["tau"])
        nde = L.iscsi_ndet()
        ce = torch.tensor(unit_vector(nde, 43), dtype=torch.float64, device="cuda")
        se = torch.empty_like(ce)
        ms = timed(ce, se)
        upd = L.iscsi_updates_per_sigma()
        st = L.iscsi_stats()
        electrons.append({"workload": ename, "norb": ew["n"], "nalpha": ew["na"], "nbeta": ew["nb"],
                          "ndet": nde, "ms_per_sigma": round(ms, 4), "updates_per_sigma": upd,
                          "gupdates_per_s": round(upd / (ms * 1e-3) / 1e9, 1),
                          "route_fp64": st.get("route_fp64")})
        L.iscsi_finalize()
    out["electron_counts"] = electrons
    return out


def run_propagation(name, nsteps=4, dt=0.02, krylov=12, with_cpu=True):
    """Real-time propagation under H(t) = H_tau + f(t) V (Eq. ham with h(t) =
    h + f(t) v, v dipole-like, f(t) = 0.05 sin(0.8 t)) by the short-iterative
    Lanczos propagator: ms per step (one warm-up step first), the sigma work
    per step, norm and energy drift, the Krylov error indicator."""
    import numpy as np
    import torch

    from paper_1609_07757_gb300 import _lib as L
    from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

    wl = WORKLOADS[name]
    n = wl["n"]
    h1, eri = make_integrals(n, wl["seed"], ell=wl["ell"], nchol=wl["nchol"], box=wl["box"])
    stream = torch.cuda.current_stream()
    L.iscsi_set_stream(stream)
    L.iscsi_init(n, wl["na"], wl["nb"], wl["kmax"], dipole_like(n), None, wl["tau"])
    hv = L.iscsi_ctx_current()
    L.iscsi_init(n, wl["na"], wl["nb"], wl["kmax"], h1, eri, wl["tau"])
    ndet, updates = L.iscsi_ndet(), L.iscsi_updates_per_sigma()
    c = torch.zeros((2, ndet), dtype=torch.float64, device="cuda")
    c[0] = torch.tensor(unit_vector(ndet, 29), dtype=torch.float64, device="cuda")
    field = 0.05 * np.sin(0.8 * dt * (np.arange(nsteps + 1) + 0.5))
    L.iscsi_propagate(c, 1, dt, field[:1], hv, krylov)  # warm-up step (work lists, routing)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    diag = L.iscsi_propagate(c, nsteps, dt, field[1:], hv, krylov)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / nsteps
    norm = float(torch.linalg.norm(c))
    route = L.iscsi_stats().get("route_fp64")
    L.iscsi_finalize()
    sig = 2 * krylov  # sigma vectors of H_k per step (complex vectors: nvec = 2; f_k V folded into H's matrices)
    out = {"workload": name, "ndet": ndet, "steps": nsteps, "dt": dt, "krylov": krylov, "ms_per_step": round(ms, 3),
           "sigma_vectors_per_step": sig,
           "effective_gupdates_per_s": round(sig * updates / (ms * 1e-3) / 1e9, 1),
           "norm_drift": abs(norm - 1.0), "max_error_indicator": float(diag[:, 0].max()),
           "energy_per_step": [round(float(x), 10) for x in diag[:, 1]],
           "field": "0.05 sin(0.8 t), position-like one-body coupling", "route_fp64": route}
    if with_cpu:
        # the oracle's row-wise sigma on a bounded sample, scaled to the sigma work of one step
        o, nrow, times, cores = cpu_baseline(wl, wl["tau"], target_s=8.0, steps=1)
        sigma_s = times[0] * o.ndet / nrow
        out["cpu_baseline"] = {"value": round(sig * sigma_s * 1e3, 1), "unit": "ms per step (extrapolated)",
                               "cores": cores, "kind": "oracle",
                               "sample": "row-wise oracle sigma on %d of %d rows (%.1f s), scaled to %d sigma "
                                         "vectors of H per step" % (
                                             nrow, o.ndet, times[0], sig)}
    return out


def context_strings(L, na, nb):
    """(alpha orbitals, alpha levels, beta orbitals, beta levels, max level sum) of the current context."""
    ga, la = L.iscsi_get_strings(0, na)
    gb, lb = L.iscsi_get_strings(1, nb)
    return ga, la, gb, lb, L.iscsi_stats()["max_excitation"]


def index_map_to_oracle(o, strings):
    """The oracle's index of every determinant of a context (its order: alpha
    strings in turn, each with the prefix of level-sorted beta strings its level
    allows); strings from context_strings, o a full-CI oracle."""
    import numpy as np
    ga, la, gb, lb, kmax = strings
    oa, _ = o.strings(0)
    ob, _ = o.strings(1)
    off = o.offsets()
    posa = {tuple(int(x) for x in r): i for i, r in enumerate(oa)}
    posb = {tuple(int(x) for x in r): i for i, r in enumerate(ob)}
    pa = np.array([posa[tuple(int(x) for x in r)] for r in ga])
    pb = np.array([posb[tuple(int(x) for x in r)] for r in gb])
    nba = np.searchsorted(lb, kmax - la, side="right")
    return np.concatenate([off[pa[a]] + pb[:nba[a]] for a in range(len(ga))])


# the paper's GAS use (Sec. "Generalized Active Space"): occupied, bound and
# continuum orbitals with at most one electron in the continuum
GAS_SPLIT = {"fci_n60": ((2, 18, 40), (0, 3, 4), (4, 4, 4))}


def run_gas(name, steps=10, warmup=3, with_cpu=True, projected=True):
    """Sigma and the ground state under a GAS restriction (P H P, at most one
    electron in the continuum subspace): ms per sigma with and without the
    restriction (L2 flushed), the projection overhead against its HBM bound,
    a Davidson ground state on the restricted space against the unrestricted
    one, sampled rows against the oracle."""
    import numpy as np
    import torch

    from paper_1609_07757_gb300 import _lib as L
    from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

    wl = WORKLOADS[name]
    sizes, cmin, cmax = GAS_SPLIT[name]
    n = wl["n"]
    h1, eri = make_integrals(n, wl["seed"], ell=wl["ell"], nchol=wl["nchol"], box=wl["box"])
    stream = torch.cuda.current_stream()
    L.iscsi_set_stream(stream)
    L.iscsi_init(n, wl["na"], wl["nb"], wl["kmax"], h1, eri, wl["tau"])
    ndet = L.iscsi_ndet()
    c = torch.tensor(unit_vector(ndet, 31), dtype=torch.float64, device="cuda")
    s = torch.empty_like(c)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(phases=False):
        for _ in range(max(3, warmup)):
            L.iscsi_sigma(c, s, 1)
        torch.cuda.synchronize()
        if phases:  # per-phase events of the timed calls only (restarts the record)
            L.iscsi_set_option("phase_timing", 1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            L.iscsi_sigma(c, s, 1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    out = {"workload": name, "subspaces": {"sizes": list(sizes), "cmin": list(cmin), "cmax": list(cmax),
                                           "meaning": "2 occupied, 18 bound, 40 continuum orbitals; at most one "
                                                      "electron in the continuum"}}
    if projected:
        ms_plain = timed()
        st, e_full = L.iscsi_davidson(1, 1e-8)
        kept = L.iscsi_set_gas(sizes, cmin, cmax)
        ms_gas = timed()
        t0 = time.time()
        st2, e_gas = L.iscsi_davidson(1, 1e-8)
        dav_s = time.time() - t0
        iters = L.iscsi_stats()["davidson_iters"]
        hbm, hbm_src = measured_peaks()
        proj_bytes = 2 * ndet * (1 + 8 + 8)  # mask + read + write, input and output
        out["projected"] = {
            "ndet": ndet, "ndet_gas": kept, "ms_per_sigma": round(ms_gas, 4),
            "ms_per_sigma_unrestricted": round(ms_plain, 4), "projection_overhead_ms": round(ms_gas - ms_plain, 4),
            "projection_hbm_bound_ms": round(proj_bytes / (hbm * 1e9) * 1e3, 4), "projection_bytes": proj_bytes,
            "hbm_peak_gbs": hbm, "peak_source": hbm_src,
            "davidson": {"status": st2, "energy_gas": float(e_gas[0]), "energy_unrestricted": float(e_full[0]),
                         "iterations": iters, "seconds": round(dav_s, 3)}}
    L.iscsi_finalize()
    # the same restriction as a GAS context: the level split at the continuum
    # (levels count continuum electrons, at most one) gives the GAS space itself
    L.iscsi_init_gas(n, wl["na"], wl["nb"], sizes, cmin, cmax, h1, eri, wl["tau"])
    st_ctx = L.iscsi_stats()
    ndet_ctx = L.iscsi_ndet()
    c = torch.tensor(unit_vector(ndet_ctx, 31), dtype=torch.float64, device="cuda")
    s = torch.empty_like(c)
    ms_ctx = timed(phases=True)
    st_t = L.iscsi_stats()
    L.iscsi_set_option("phase_timing", 0)
    upd_ctx = L.iscsi_updates_per_sigma()
    s_ctx = s.cpu().numpy()
    t0 = time.time()
    st3, e_ctx = L.iscsi_davidson(1, 1e-8)
    dav_ctx_s = time.time() - t0
    iters_ctx = L.iscsi_stats()["davidson_iters"]
    strings = context_strings(L, wl["na"], wl["nb"])
    L.iscsi_finalize()
    # the dominant kernel of the GAS context's sigma, timed live (phase events)
    gemm_ms = st_t["phase_ms"]["opposite_gemm"] / max(1, st_t["timed_calls"])
    both = st_t.get("both_tc_fp64", 0) == 1
    route = st_t.get("route_fp64", {})
    if st_t.get("fp64_tc", 0) == 1 and route.get("ab_tc", 1) == 1 and gemm_ms > 0:
        flops = st_t["opposite_tc_bf16_flops"] + (st_t.get("samespin_tc_bf16_flops", 0.0) if both else 0.0)
        peak, peak_src = bf16_peak()
        ach = flops / (gemm_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": round(ach, 4), "peak": peak, "unit": "TFLOP/s",
                "frac": round(ach / peak, 4),
                "traffic": profile_traffic("k_oz_gemm%s_gas_%s" % ("_both" if both else "", name))[0],
                "kernel": "k_oz_gemm (tcgen05, FP64-accurate, %s)" % (
                    "opposite- and same-spin contractions in one launch" if both else "opposite-spin"),
                "kernel_ms": round(gemm_ms, 4), "flops_per_launch": flops, "peak_source": peak_src}
    else:
        roof = {"bound": None, "note": "opposite-spin contraction not on the tensor cores", "route": route}
    out.update({
           "gas_context": {"ndet": ndet_ctx, "level_split": st_ctx["level_split"],
                           "max_excitation": st_ctx["max_excitation"], "mask": st_ctx["gas_subspaces"] > 0,
                           "ms_per_sigma": round(ms_ctx, 4), "gupdates_per_s": round(upd_ctx / (ms_ctx * 1e-3) / 1e9, 1),
                           "speedup_vs_projected": round(ms_gas / ms_ctx, 2) if projected else None,
                           "roofline": roof, "route_fp64": route,
                           "davidson": {"status": st3, "energy": float(e_ctx[0]), "iterations": iters_ctx,
                                        "seconds": round(dav_ctx_s, 3),
                                        "abs_dE_vs_projected": abs(float(e_ctx[0]) - float(e_gas[0]))
                                        if projected else None}},
           "l2": "flushed between calls",
           "note": "projected: sigma on the enclosing full-CI space with the mask; gas_context: iscsi_init_gas, "
                   "whose level split makes the GAS space the computed space"})
    if with_cpu:
        # the full-CI oracle on sampled rows of the GAS space (the GAS context's
        # vector mapped to full-CI indices), calibrated to ~5 s, scaled to all rows
        from oracle import Oracle, gas, max_threads
        o = Oracle(n, wl["na"], wl["nb"], 99, wl["tau"], h1, eri)
        keep = gas.mask(o, sizes, cmin, cmax)
        idx = index_map_to_oracle(o, strings)
        c_or = np.zeros(o.ndet)
        c_or[idx] = unit_vector(len(idx), 31)
        rng = np.random.default_rng(2)
        m = 64
        for _ in range(3):
            rows = rng.choice(len(idx), size=min(m, len(idx)), replace=False)
            t0 = time.time()
            ref = o.sigma_rows(c_or, idx[rows])
            dt = time.time() - t0
            if dt >= 2.5 or m >= len(idx):
                break
            m = int(min(len(idx), m * 5.0 / max(dt, 1e-3)))
        out["sample_check"] = {"rows": len(rows), "max_abs_diff": float(np.abs(s_ctx[rows] - ref).max()),
                               "scale": float(np.abs(s_ctx).max()),
                               "gas_ndet_equal": bool(int(keep.sum()) == len(idx))}
        out["cpu_baseline"] = {"value": round(dt / len(rows) * len(idx) * 1e3, 1),
                               "unit": "ms per sigma (extrapolated)", "cores": max_threads(), "kind": "oracle",
                               "sample": "row-wise full-CI oracle sigma on %d GAS rows (%.2f s), scaled to the %d "
                                         "GAS rows" % (len(rows), dt, len(idx))}
    return out


def run_sweep(steps=5, warmup=3):
    """The box-size sweep: CISD and CISDT, 2 alpha + 2 beta electrons in 50, 100,
    150 and 200 orbitals (integrals decaying with the box), tau = 1e-14, FP64.
    sigma time per orbital count and the exponent of a least-squares fit
    t ~ n^p over the four sizes."""
    import math

    import torch

    from paper_1609_07757_gb300 import _lib as L
    from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

    out = {}
    for k, name in ((2, "cisd"), (3, "cisdt")):
        rows = []
        for n in (50, 100, 150, 200):
            wl = WORKLOADS["%s_n%d" % (name, n)]
            h1, eri = make_integrals(wl["n"], wl["seed"], ell=wl["ell"], nchol=wl["nchol"], box=wl["box"])
            L.iscsi_init(wl["n"], wl["na"], wl["nb"], wl["kmax"], h1, eri, wl["tau"])
            nd = L.iscsi_ndet()
            c = torch.tensor(unit_vector(nd, 11), dtype=torch.float64, device="cuda")
            sg = torch.empty_like(c)
            for _ in range(warmup):
                L.iscsi_sigma(c, sg, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(steps):
                L.iscsi_sigma(c, sg, 1)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            st = L.iscsi_stats()
            upd = L.iscsi_updates_per_sigma()
            kept = st["units_kept_opposite"] / max(1, st["units_total"]["opposite"])
            rows.append({"norb": n, "ndet": nd, "sigma_ms": round(ms, 3), "GUpdates_per_s": round(upd / ms / 1e6, 1),
                         "updates": upd, "opposite_units_kept": round(kept, 4)})
            L.iscsi_finalize()
        xs = [math.log(r["norb"]) for r in rows]
        ys = [math.log(r["sigma_ms"]) for r in rows]
        yu = [math.log(r["updates"]) for r in rows]
        mx = sum(xs) / len(xs)

        def slope(y):
            my = sum(y) / len(y)
            return sum((a - mx) * (b - my) for a, b in zip(xs, y)) / sum((a - mx) ** 2 for a in xs)
        out[name] = {"points": rows, "time_exponent": round(slope(ys), 3), "updates_exponent": round(slope(yu), 3)}
    return out


def cpu_baseline(wl, tau, target_s=15.0, steps=1):
    """The oracle, as it stands, on a bounded sample of rows of the same workload."""
    import numpy as np

    import oracle
    from paper_1609_07757_gb300.synthetic import make_integrals, unit_vector

    h1, eri = make_integrals(wl["n"], wl["seed"], ell=wl["ell"], nchol=wl["nchol"], box=wl["box"])
    o = oracle.Oracle(wl["n"], wl["na"], wl["nb"], wl["kmax"], tau, h1, eri)
    c = unit_vector(o.ndet, 17)
    rng = np.random.default_rng(5)
    cores = oracle.max_threads()
    # calibrate the sample size on a few rows, then on a sample a tenth of the target
    nrow = min(o.ndet, 4 * cores)
    for target in (0.1 * target_s, target_s):
        rows = rng.choice(o.ndet, size=nrow, replace=False)
        t0 = time.time()
        o.sigma_rows(c, rows)
        per_row = max((time.time() - t0) / len(rows), 1e-7)
        nrow = int(min(o.ndet, max(len(rows), target / per_row)))
    times = []
    for _ in range(steps):
        rows = rng.choice(o.ndet, size=nrow, replace=False)
        t0 = time.time()
        o.sigma_rows(c, rows)
        times.append(time.time() - t0)
    return o, nrow, times, cores


def run_reference(args, wl, ws, rank):
    tau = args.tau if args.tau is not None else wl["tau"]
    if rank != 0:
        return None
    total_s = 150.0
    per_step = max(2.0, total_s / max(1, args.steps + args.warmup))
    o, nrow, times, cores = cpu_baseline(wl, tau, target_s=per_step, steps=args.steps + args.warmup)
    times = times[args.warmup:]
    upd = args.updates
    frac = nrow / o.ndet
    mean_s = sum(times) / len(times)
    value = upd * frac / mean_s / 1e9 if upd else None
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 6) if value else None,
        "unit": "GUpdates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(mean_s * 1e3 / frac, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "norb": wl["n"], "ndet": o.ndet, "tau": tau},
        "cpu_baseline": {"value": round(value, 6) if value else None, "unit": "GUpdates/s", "cores": cores,
                         "kind": "oracle",
                         "sample": "row-wise oracle sigma on %d of %d rows per step, scaled by the row fraction"
                                   % (nrow, o.ndet)},
        "e2e": {"value": round(value, 6) if value else None, "unit": "GUpdates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fci_n60", choices=sorted(WORKLOADS))
    ap.add_argument("--tau", type=float, default=None)
    ap.add_argument("--precision", type=int, default=64, choices=[32, 64])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mixed-workload", default="fci_n100", choices=sorted(WORKLOADS) + ["none"],
                    help="workload of the FP32-mixed vs FP64 Davidson comparison added to the line")
    ap.add_argument("--mixed-roots", type=int, default=3)
    ap.add_argument("--roots", type=int, default=2,
                    help="lowest roots of the main workload by Davidson, pinned to the oracle (0: skip)")
    ap.add_argument("--oracle-full", action="store_true",
                    help="pin the roots with a full oracle sigma (minutes) instead of a sample of rows")
    ap.add_argument("--tau-sweep", type=int, default=1, choices=[0, 1],
                    help="time sigma at the workload's other screening thresholds")
    ap.add_argument("--batching", type=int, default=16, metavar="COUNT",
                    help="the batching form: COUNT full-CI instances, batched vs one at a time (0: off)")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="library option autotune (kernel routing timed at the first sigma)")
    ap.add_argument("--density-workload", default="fci_n60", choices=sorted(WORKLOADS) + ["none"],
                    help="one- and two-body density matrices on this workload (none: skip)")
    ap.add_argument("--propagation-workload", default="fci_n60", choices=sorted(WORKLOADS) + ["none"],
                    help="real-time propagation under a field on this workload (none: skip)")
    ap.add_argument("--gas-workload", default="fci_n60", choices=sorted(GAS_SPLIT) + ["none"],
                    help="sigma and ground state under a GAS restriction on this workload (none: skip)")
    ap.add_argument("--operators-workload", default="fci_n60", choices=sorted(WORKLOADS) + ["none"],
                    help="operators other than H (transition, dipole, dipole squared) and sigma at 3 and 4 "
                         "electrons per spin")
    ap.add_argument("--operators-only", action="store_true", help="run only the operators leg and print its object")
    ap.add_argument("--gas-only", action="store_true", help="run only the GAS leg and print its object")
    ap.add_argument("--gas-context-only", action="store_true",
                    help="with --gas-only: only the GAS context (iscsi_init_gas), not the projected form")
    ap.add_argument("--propagation-only", action="store_true",
                    help="run only the propagation leg (--steps steps) and print its object")
    ap.add_argument("--density-only", action="store_true",
                    help="run only the density-matrix leg and print its object")
    ap.add_argument("--sweep", type=int, default=1, choices=[0, 1],
                    help="the CISD/CISDT box-size sweep (n = 50..200) with its fitted scaling exponents")
    ap.add_argument("--updates", type=float, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    ws, rank, local = dist_env()
    wl = WORKLOADS[args.workload]
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        if args.updates is None:
            # the oracle's own count of the workload's updates per sigma (oracle/counts.py)
            from oracle.counts import updates_per_sigma
            from paper_1609_07757_gb300.synthetic import make_integrals
            tau = args.tau if args.tau is not None else wl["tau"]
            h1, eri = make_integrals(wl["n"], wl["seed"], ell=wl["ell"], nchol=wl["nchol"], box=wl["box"])
            args.updates = updates_per_sigma(wl["n"], wl["na"], wl["nb"], wl["kmax"], tau, h1, eri)
        line = run_reference(args, wl, ws, rank)
        if rank == 0 and line:
            print(json.dumps(line))
        return
    if args.operators_only:
        if rank == 0:
            from paper_1609_07757_gb300 import _lib as L
            L.iscsi_set_option("autotune", args.autotune)
            print(json.dumps({"operators": run_operators(args.operators_workload, steps=args.steps,
                                                         warmup=args.warmup)}))
        return
    if args.propagation_only or args.density_only or args.gas_only:
        from paper_1609_07757_gb300 import _lib as L
        L.iscsi_set_option("autotune", args.autotune)
    if args.propagation_only:
        # the propagation leg alone (profiling its launches)
        if rank == 0:
            print(json.dumps({"propagation": run_propagation(args.propagation_workload, nsteps=args.steps,
                                                             with_cpu=not args.no_cpu_baseline)}))
        return
    if args.gas_only:
        if rank == 0:
            print(json.dumps({"gas": run_gas(args.gas_workload, steps=args.steps, warmup=args.warmup,
                                             with_cpu=not args.no_cpu_baseline,
                                             projected=not args.gas_context_only)}))
        return
    if args.density_only:
        # the density-matrix leg alone (profiling its contraction)
        if rank == 0:
            print(json.dumps({"density_matrices": run_density(args.density_workload, steps=args.steps,
                                                              warmup=args.warmup,
                                                              with_cpu=not args.no_cpu_baseline)}))
        return
    line = run_ours(args, wl, ws, rank, local)
    if rank == 0 and ws == 1 and args.mixed_workload != "none":
        # the precision form: FP32-mixed vs FP64 Davidson, |dE| and speedup (untimed by the contract)
        line["mixed_precision"] = run_precision_form(args.mixed_workload, args.mixed_roots,
                                                     with_oracle=not args.no_cpu_baseline)
    if args.batching > 0:
        # every rank runs its share of the instances; rank 0 reports the job
        b = run_batching(args.batching, rank=rank, ws=ws)
        if rank == 0:
            line["batching"] = b
    if rank == 0 and ws == 1 and args.sweep:
        line["box_sweep"] = run_sweep()
    if rank == 0 and ws == 1 and args.density_workload != "none":
        line["density_matrices"] = run_density(args.density_workload, with_cpu=not args.no_cpu_baseline)
    if rank == 0 and ws == 1 and args.propagation_workload != "none":
        line["propagation"] = run_propagation(args.propagation_workload, with_cpu=not args.no_cpu_baseline)
    if rank == 0 and ws == 1 and args.gas_workload != "none":
        line["gas"] = run_gas(args.gas_workload, with_cpu=not args.no_cpu_baseline)
    if rank == 0 and ws == 1 and args.operators_workload != "none":
        line["operators"] = run_operators(args.operators_workload)
    if rank == 0:
        if not args.no_cpu_baseline and ws == 1:
            tau = args.tau if args.tau is not None else wl["tau"]
            o, nrow, times, cores = cpu_baseline(wl, tau, target_s=15.0, steps=1)
            frac = nrow / o.ndet
            val = line["config"]["updates_per_sigma"] * frac / times[0] / 1e9
            line["cpu_baseline"] = {"value": round(val, 6), "unit": "GUpdates/s", "cores": cores, "kind": "oracle",
                                    "sample": "row-wise oracle sigma on %d random rows of %d (%.1f s), scaled by "
                                              "the row fraction" % (nrow, o.ndet, times[0])}
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
