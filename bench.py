"""Benchmark of the Q-less QR hot path on GB300 (one JSON line on stdout, rank 0).

Workload (one "step"): the single-matrix condition sweep -- X = G S with m = 2^25 rows,
n in {1, 2, 4, 8, 16, 32, 64}, kappa = 1e4, FP64 storage, each X factored by Q-less TSQR,
Cholesky-QR2 and SVQB2.  Inputs are device-resident before the timed region and every X is
larger than the 129 MB L2 (>= 268 MB), so no L2 flush is needed between steps.

metric: effective GB/s = sum over calls of 8 m n bytes / sum of the calls' time (the
paper's "effective bandwidth", counted once per call even though the Gram methods read X
twice).  Per-call breakdown, the roofline of the dominant kernel, the oracle on the host
cores, the host-buffer end-to-end number and the SM clocks seen during the timed region
are attached.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
N > 1 runs under torch.distributed.run: every rank factors the same sweep on its own GPU
(independent replicas; the method has no cross-GPU exchange in this build).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M = 1 << 25
NS = [1, 2, 4, 8, 16, 32, 64]
LS_M, LS_N = 1 << 24, 31  # least-squares [A b] workload
KAPPA = 1e4
METHODS = ["tsqr", "cholqr2", "svqb2"]
PASSES = {"tsqr": 1, "cholqr2": 2, "svqb2": 2}
# DRAM bytes (read + write) per row of X per launch, from one ncu capture of the same kernel
# on a smaller m (dram__bytes_read.sum + dram__bytes_write.sum of that launch / its m); the
# roofline's "traffic" is this times m for the dominant call, null where no capture of the
# current kernel exists.
MEASURED_TRAFFIC_PER_ROW = {
    ("tsqr", 64): (1.074413e9 + 3.693568e6) / 2 ** 21,       # tsqr_kernel<64, 16, 16, 256>, m = 2^21
    ("tsqr", 4): (536.98944e6 + 3.195648e6) / 2 ** 24,       # tsqr_kernel<4, 1, 8, 128>, m = 2^24
    ("cholqr2", 64): (2.256619e9 + 174.161664e6) / 2 ** 22,  # gram_pipe_kernel<64> (first pass), m = 2^22
}


# FP32 instructions of one double-float (dot, update) pair of the Householder column step:
# an accumulating product (13, lo * lo kept) and a product subtracted with renormalisation (15)
DF_INSTR_PER_PAIR = 28


def rel_err(R, R_ref) -> float:
    """||R - R_ref||_F / ||R_ref||_F, the accuracy measure of the batched and serving checks."""
    import numpy as np

    R, R_ref = np.asarray(R, dtype=np.float64), np.asarray(R_ref, dtype=np.float64)
    den = float(np.linalg.norm(R_ref))
    return float(np.linalg.norm(R - R_ref)) / (den if den > 0 else 1.0)


def row_err(R, R_ref) -> float:
    """max_ij |R_ij - R_ref_ij| / |R_ref_ii| over the upper triangle (rows with a zero
    reference diagonal scaled by ||R_ref||_F): every entry against its row's diagonal."""
    import numpy as np

    R, R_ref = np.asarray(R, dtype=np.float64), np.asarray(R_ref, dtype=np.float64)
    fro = float(np.linalg.norm(R_ref)) or 1.0
    d = np.abs(np.diag(R_ref)).copy()
    d[d == 0] = fro
    D = np.triu(np.abs(R - R_ref)) / d[:, None]
    return float(D.max()) if D.size else 0.0


def tolerance(n: int, kappa: float) -> float:
    """The stated bound on rel_err for FP64 TSQR: 1e-13 n kappa(X)."""
    return 1e-13 * n * max(float(kappa), 1.0)


def lapack_r(X):
    """R of X (m x n, host) from LAPACK's Householder QR, rows scaled to a nonnegative diagonal."""
    import numpy as np

    R = np.linalg.qr(np.asarray(X, dtype=np.float64), mode="r")
    sg = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    return R * sg[:, None]


def kernel_name(meth: str, n: int) -> str:
    if meth == "tsqr":
        return "tsqr_kernel"
    return "gram_umma_kernel" if n > 32 else ("gram_tc_kernel" if n > 8 else "gram_kernel")
METRIC = "Q-less QR effective GB/s (8mn B/time)"
WORKLOAD = ("Q-less QR condition sweep: X = G S, m = 2^25 rows, n in {1,2,4,8,16,32,64}, kappa = 1e4, "
            "FP64 storage; TSQR + Cholesky-QR2 + SVQB2 per n; plus least squares via the QR of [A b], "
            "A 2^24 x 31 (kappa 1e3), FP64- and FP32-stored")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    # the first end-to-end step fills the copy pipeline (nothing to overlap its copies with,
    # and host -> device copies run at a fraction of the link rate while the GPU idles):
    # ten steps spread that fill the way a long run does
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-batched", dest="batched", action="store_false")
    p.add_argument("--no-serving", dest="serving", action="store_false")
    p.add_argument("--no-cpu-context", dest="cpu_context", action="store_false",
                   help="skip the all-core torch.linalg.qr context number")
    p.add_argument("--no-accuracy", dest="accuracy", action="store_false",
                   help="skip the full-size accuracy check of the default arithmetic against native FP64")
    p.add_argument("--no-next", dest="next_rows", action="store_false",
                   help="skip the measurements of the rows beyond the sweep (shifted Cholesky-QR3, Q = X R^-1, "
                        "two-phase orthogonalisation, n > 64)")
    p.add_argument("--case", default=None,
                   help="METHOD:N:M -- time one call shape alone (profiling aid; prints its own JSON line)")
    return p.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ multi-rank aggregation


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(bytes_per_step: float, steps: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: every rank processed bytes_per_step per step (weak scaling);
    the job took the slowest rank's time."""
    return world * bytes_per_step * steps / (max_ms / 1e3) / 1e9


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ our arm


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2603_20889_gb300 as q
    from paper_2603_20889_gb300 import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    lib = q.load_library()
    stream = torch.cuda.current_stream()
    sptr = q._stream_ptr(stream)

    # inputs resident in HBM before the timed region
    Xs = {n: synth.conditioned_device(M, n, KAPPA, seed=1000 + n, device=dev) for n in NS}
    nmax = max(NS)
    wsb = max(lib.ql_workspace_bytes(q.QL_AUTO, M, n, q.QL_F64) for n in NS)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    Rb = {n: torch.empty((n, n), dtype=torch.float64, device=dev) for n in NS}

    def call(method, n, X, R, inf):
        ptr = X.data_ptr()
        if method == "tsqr":
            st = lib.ql_tsqr_qless(M, n, ptr, q.QL_F64, M, R.data_ptr(), n, inf.data_ptr(), ws.data_ptr(), wsb, sptr)
        elif method == "cholqr2":
            st = lib.ql_cholqr2_qless(M, n, ptr, q.QL_F64, M, R.data_ptr(), n, inf.data_ptr(), ws.data_ptr(), wsb,
                                      sptr)
        else:
            st = lib.ql_svqb_qless(M, n, ptr, q.QL_F64, M, R.data_ptr(), n, None, 0.0, inf.data_ptr(),
                                   ws.data_ptr(), wsb, sptr)
        if st != 0:
            raise RuntimeError(f"{method} n={n}: status {st}")

    calls = [(meth, n) for n in NS for meth in METHODS] + [("lstsq_f64", LS_N), ("lstsq_f32", LS_N)]
    # least squares through the QR of [A b]: A 2^24 x 31 (kappa 1e3), b = A x* + 1e-6 noise,
    # FP64- and FP32-stored
    import numpy as np

    At = synth.conditioned_device(LS_M, LS_N, 1e3, seed=4242, device=dev)
    xs = torch.from_numpy(np.random.default_rng(4243).standard_normal(LS_N)).to(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(4244)
    bvec = xs @ At + 1e-6 * torch.randn(LS_M, generator=g, device=dev, dtype=torch.float64)
    ls = {"lstsq_f64": (At, bvec, q.QL_F64), "lstsq_f32": (At.float(), bvec.float(), q.QL_F32)}
    xout = torch.empty(LS_N + 1, dtype=torch.float64, device=dev)

    def call_ls(name, inf):
        A, b, dt = ls[name]
        st = lib.ql_lstsq_qless(LS_M, LS_N, A.data_ptr(), LS_M, b.data_ptr(), dt, q.QL_TSQR, xout.data_ptr(),
                                xout[LS_N:].data_ptr(), None, inf.data_ptr(), ws.data_ptr(), wsb, sptr)
        if st != 0:
            raise RuntimeError(f"{name}: status {st}")

    def nbytes(meth, n):
        if meth == "lstsq_f64":
            return 8.0 * LS_M * (n + 1)
        if meth == "lstsq_f32":
            return 4.0 * LS_M * (n + 1)
        return 8.0 * M * n

    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in calls]
           for _ in range(args.steps)]
    info = torch.zeros((len(calls), 2), dtype=torch.int32, device=dev)

    def step(ev=None):
        for i, (meth, n) in enumerate(calls):
            if ev:
                ev[i][0].record(stream)
            if meth.startswith("lstsq"):
                call_ls(meth, info[i])
            else:
                call(meth, n, Xs[n], Rb[n], info[i])
            if ev:
                ev[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    bad = [(calls[i], v) for i, v in enumerate(info.cpu().tolist()) if v[0] != 0]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    per_call = [0.0] * len(calls)
    l0 = lib.ql_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    for k in range(args.steps):  # per-call device times (events on the launching stream)
        for i in range(len(calls)):
            per_call[i] += evs[k][i][0].elapsed_time(evs[k][i][1])
    launches = lib.ql_launch_count() - l0
    if world > 1:
        torch.distributed.barrier()
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), dev)
    clk = clocks.stop()

    bytes_step = sum(nbytes(meth, n) for (meth, n) in calls)
    ms_step = total_ms / args.steps
    value = whole_job_gbs(bytes_step, args.steps, world, total_ms)

    # dominant call (largest share of the step) and its roofline (HBM, algorithmic bytes)
    peak, peak_kind = measured_peaks()
    sweep = []
    for i, (meth, n) in enumerate(calls):
        ms = per_call[i] / args.steps
        sweep.append({"method": meth, "n": n, "ms": round(ms, 4), "eff_gbs": round(nbytes(meth, n) / ms / 1e6, 1),
                      "alg_gbs": round(PASSES.get(meth, 1) * nbytes(meth, n) / ms / 1e6, 1)})
    dom = max(range(len(calls)), key=lambda i: per_call[i])
    dmeth, dn = calls[dom]
    dms = per_call[dom] / args.steps
    # the timed share of the dominant kernel: one pass = one launch reading its bytes
    kern_ms = dms / PASSES.get(dmeth, 1)
    achieved = nbytes(dmeth, dn) / kern_ms / 1e6
    per_row = MEASURED_TRAFFIC_PER_ROW.get((dmeth, dn))
    traffic = int(per_row * M) if per_row else None
    hbm_view = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_kind}
    kname = f"{kernel_name(dmeth, dn)} ({dmeth}, n={dn}, m=2^25)"
    # measured compute-pipe peaks of this GPU (FP32 / FP64 FMA, FP64 MMA, the library's
    # double-float multiply-accumulate), the denominators of the arithmetic-bound rooflines
    try:
        peaks = {k: round(v, 3) for k, v in q.measure_peaks(stream).items()}
        peaks["unit"] = "TFLOP/s"
    except Exception as exc:
        peaks = {"error": repr(exc)[:200]}
    if dmeth == "tsqr" and dn > 1:
        # the double-float Householder is bound by the FP32 pipes: 2 m n^2 FP64-equivalent
        # flops per launch against the measured FP32 FMA instruction rate at 27 FP32
        # instructions per (dot, update) pair of 4 flops
        flops = 2.0 * M * dn * dn
        ach = flops / (kern_ms / 1e3) / 1e12
        if "fp32_fma" in peaks:
            alu_peak = peaks["fp32_fma"] / 2.0 * 4.0 / DF_INSTR_PER_PAIR
            src = "measured"
            deriv = (f"measured FP32 FMA rate {peaks['fp32_fma']} TFLOP/s = {peaks['fp32_fma'] / 2:.2f} T instr/s, "
                     f"x 4 FP64-equivalent flops per {DF_INSTR_PER_PAIR} FP32 instructions (one dot + update pair)")
        else:
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            clk_hz = float(clk.get("sm_max_mhz") or 2070.0) * 1e6
            alu_peak = sms * 128 * clk_hz / (DF_INSTR_PER_PAIR / 4.0) / 1e12
            src = "derived"
            deriv = (f"{sms} SMs x 128 FP32 lanes x {clk_hz / 1e6:.0f} MHz / "
                     f"({DF_INSTR_PER_PAIR} FP32 instructions per 4 FP64-equivalent flops)")
        roofline = {"bound": "alu", "achieved": round(ach, 3), "peak": round(alu_peak, 3), "unit": "TFLOP/s",
                    "frac": round(ach / alu_peak, 4), "traffic": traffic, "peak_source": src,
                    "peak_derivation": deriv,
                    "kernel": kname, "algorithmic_flops_per_launch": int(flops),
                    "algorithmic_bytes_per_launch": int(nbytes(dmeth, dn)), "hbm": hbm_view,
                    "note": "per-launch time from CUDA events around the call on its stream"}
    else:
        roofline = dict(hbm_view, traffic=traffic, kernel=kname,
                        algorithmic_bytes_per_launch=int(nbytes(dmeth, dn)),
                        note="per-launch time from CUDA events around the call on its stream; Gram methods: "
                             "call time / 2 passes")

    e2e = run_e2e(args, q, lib, torch, dev, Xs, ws, wsb, stream, ls, world) if args.e2e_steps > 0 else None
    accuracy = None
    if args.accuracy:
        try:
            accuracy = run_accuracy(q, lib, torch, dev, stream, Xs)
        except Exception as exc:
            accuracy = {"error": repr(exc)[:300]}
        torch.cuda.empty_cache()
    del ls, At, bvec
    del Xs
    torch.cuda.empty_cache()
    extra = {}
    if args.next_rows:
        try:
            extra["scholqr3"] = run_scholqr3(q, lib, torch, dev, stream)
        except Exception as exc:
            extra["scholqr3"] = {"error": repr(exc)[:300]}
        torch.cuda.empty_cache()
        try:
            extra["kappa_rows"] = run_kappa_rows(q, lib, torch, dev, stream)
        except Exception as exc:
            extra["kappa_rows"] = {"error": repr(exc)[:300]}
        torch.cuda.empty_cache()
        try:
            extra["q_from_r"] = run_qform(q, lib, torch, dev, stream)
        except Exception as exc:
            extra["q_from_r"] = {"error": repr(exc)[:300]}
        torch.cuda.empty_cache()
        try:
            extra["project_out"] = run_project(q, lib, torch, dev, stream)
        except Exception as exc:
            extra["project_out"] = {"error": repr(exc)[:300]}
        torch.cuda.empty_cache()
        try:
            extra["qr_wide"] = run_wide(q, lib, torch, dev, stream)
        except Exception as exc:
            extra["qr_wide"] = {"error": repr(exc)[:300]}
        torch.cuda.empty_cache()
    if args.batched:
        try:
            extra["batched"] = run_batched(q, lib, torch, dev, stream)
        except Exception as exc:  # reported, not fatal for the headline line
            extra["batched"] = {"error": repr(exc)[:300]}
        torch.cuda.empty_cache()
    if args.serving:
        try:
            extra["serving"] = run_serving(q, lib, torch, dev)
        except Exception as exc:
            extra["serving"] = {"error": repr(exc)[:300]}
        torch.cuda.empty_cache()
        # the same stream below the sustained rate: latencies without an ever-growing queue
        try:
            extra["serving_300"] = run_serving(q, lib, torch, dev, count=3000, rate=300.0)
        except Exception as exc:
            extra["serving_300"] = {"error": repr(exc)[:300]}
        torch.cuda.empty_cache()
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2", "data": "synthetic",
        "config": {"workload": WORKLOAD, "storage": "f64", "arith": "double-float (f32x2) m-loops, FP64 n x n",
                   "m": M, "n": NS, "kappa": KAPPA, "methods": METHODS, "parallelism": f"replicas x{world}",
                   "l2": "every input > L2 (>= 268 MB); no flush needed"},
        "roofline": roofline, "clocks": clk, "gpu_launches": int(launches),
        "gpu_launches_per_step": int(launches) // max(args.steps, 1),
        "sweep": sweep, "status_errors": bad, "compute_peaks": peaks,
    }
    if e2e:
        out["e2e"] = e2e
    if accuracy:
        out["accuracy"] = accuracy
    out.update(extra)
    return out


def run_e2e(args, q, lib, torch, dev, Xs, ws, wsb, stream, ls, world=1):
    """The same sweep through the C ABI from HOST buffers: every step copies each X from
    pinned host memory to the device (two copy streams, one device buffer per matrix, so
    copies overlap the factorisations still running) and reads every R back, all inside
    the timed region."""
    import torch as _t

    host = {n: _t.empty(Xs[n].shape, dtype=Xs[n].dtype, pin_memory=True) for n in NS}
    for n in NS:
        host[n].copy_(Xs[n])
    # one device buffer per matrix: the next step's copy of X_n waits only for this step's
    # factorisations of X_n, so the small matrices of step k + 1 arrive while step k's
    # widest ones are factored (copies run at full link speed only while the GPU is busy)
    bufd = {n: _t.empty(Xs[n].numel(), dtype=_t.float64, device=dev) for n in NS}
    Rh = {n: _t.empty((n, n), dtype=_t.float64, pin_memory=True) for n in NS}
    Rd = {n: _t.empty((n, n), dtype=_t.float64, device=dev) for n in NS}
    inf = _t.zeros(2, dtype=_t.int32, device=dev)
    sptr = q._stream_ptr(stream)
    # two copy streams, 1 GB pieces alternating between them: one stream of host -> device
    # copies ran at ~85 GB/s on this machine, two at the full ~211 GB/s of the link
    cstreams = [_t.cuda.Stream(device=dev), _t.cuda.Stream(device=dev)]
    copied = {n: [_t.cuda.Event(), _t.cuda.Event()] for n in NS}  # [matrix][copy stream]
    used = {n: _t.cuda.Event() for n in NS}
    hls = {k: (_t.empty(A.shape, dtype=A.dtype, pin_memory=True).copy_(A),
               _t.empty(b.shape, dtype=b.dtype, pin_memory=True).copy_(b), _t.empty_like(A), _t.empty_like(b), dt)
           for k, (A, b, dt) in ls.items()}
    xh = _t.empty(LS_N + 1, dtype=_t.float64, pin_memory=True)
    xd = _t.empty(LS_N + 1, dtype=_t.float64, device=dev)
    h2d = sum(host[n].numel() * 8 for n in NS) + sum(v[0].numel() * v[0].element_size() + v[1].numel() *
                                                     v[1].element_size() for v in hls.values())
    d2h = sum(Rh[n].numel() * 8 * len(METHODS) for n in NS) + len(hls) * (LS_N + 1) * 8
    ls_copied = {k: [_t.cuda.Event(), _t.cuda.Event()] for k in hls}
    ls_used = {k: _t.cuda.Event() for k in hls}

    def copy_in(dst, src):
        """Host -> device in pieces of at most 1 GB alternating over the two copy streams; at
        least two pieces, so that both streams carry every matrix (a matrix's factorisations
        wait for its last piece)."""
        d, h = dst.view(-1), src.reshape(-1)
        pieces = max(2, -(-h.numel() * h.element_size() // (1 << 30)))
        ch = -(-h.numel() // pieces)
        for k, i in enumerate(range(0, h.numel(), ch)):
            with _t.cuda.stream(cstreams[k % 2]):
                d[i:i + ch].copy_(h[i:i + ch], non_blocking=True)

    def copies_wait(ev):
        for cs in cstreams:
            cs.wait_event(ev)

    def copies_done(evs):
        for cs, e in zip(cstreams, evs):
            e.record(cs)
            stream.wait_event(e)

    def step(copy_per_call=False):
        for n in NS:
            dst = bufd[n]
            copies_wait(used[n])
            copy_in(dst, host[n])
            copies_done(copied[n])
            X = dst.data_ptr()
            for mi, meth in enumerate(METHODS):
                if copy_per_call and mi > 0:  # every call brings its own copy of X from the host
                    used[n].record(stream)
                    copies_wait(used[n])
                    copy_in(dst, host[n])
                    copies_done(copied[n])
                if meth == "tsqr":
                    lib.ql_tsqr_qless(M, n, X, q.QL_F64, M, Rd[n].data_ptr(), n, inf.data_ptr(), ws.data_ptr(), wsb, sptr)
                elif meth == "cholqr2":
                    lib.ql_cholqr2_qless(M, n, X, q.QL_F64, M, Rd[n].data_ptr(), n, inf.data_ptr(), ws.data_ptr(),
                                         wsb, sptr)
                else:
                    lib.ql_svqb_qless(M, n, X, q.QL_F64, M, Rd[n].data_ptr(), n, None, 0.0, inf.data_ptr(),
                                      ws.data_ptr(), wsb, sptr)
                Rh[n].copy_(Rd[n], non_blocking=True)
            used[n].record(stream)
        for name, (Ah, bh, Ad, bd, dt) in hls.items():  # least squares: [A b] from host, x back
            copies_wait(ls_used[name])  # queued behind the sweep's copies: overlaps its last factorisations
            copy_in(Ad, Ah)
            copy_in(bd, bh)
            for cs, e in zip(cstreams, ls_copied[name]):
                e.record(cs)
        for name, (Ah, bh, Ad, bd, dt) in hls.items():
            for e in ls_copied[name]:
                stream.wait_event(e)
            lib.ql_lstsq_qless(LS_M, LS_N, Ad.data_ptr(), LS_M, bd.data_ptr(), dt, q.QL_TSQR, xd.data_ptr(),
                               xd[LS_N:].data_ptr(), None, inf.data_ptr(), ws.data_ptr(), wsb, sptr)
            ls_used[name].record(stream)
            xh.copy_(xd, non_blocking=True)

    step()
    _t.cuda.synchronize()
    e0, e1 = _t.cuda.Event(enable_timing=True), _t.cuda.Event(enable_timing=True)
    e0.record(stream)
    copies_wait(e0)
    for _ in range(args.e2e_steps):
        step()
    for cs in cstreams:
        stream.wait_stream(cs)
    e1.record(stream)
    _t.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.e2e_steps
    if world > 1:  # replicas: the slowest rank's time, every rank's bytes
        _t.distributed.barrier()
        ms = max_over_ranks(ms, dev)
    bytes_step = world * (sum(8.0 * M * n * len(METHODS) for n in NS) + 12.0 * LS_M * (LS_N + 1))
    # the same calls, each bringing its own copy of X from the host (a caller that factors
    # one host matrix per call): three times the host -> device bytes per step
    steps_pc = max(2, args.e2e_steps // 3)
    step(True)
    _t.cuda.synchronize()
    e0.record(stream)
    copies_wait(e0)
    for _ in range(steps_pc):
        step(True)
    for cs in cstreams:
        stream.wait_stream(cs)
    e1.record(stream)
    _t.cuda.synchronize()
    ms_pc = e0.elapsed_time(e1) / steps_pc
    if world > 1:
        _t.distributed.barrier()
        ms_pc = max_over_ranks(ms_pc, dev)
    h2d_pc = h2d + sum(host[n].numel() * 8 for n in NS) * (len(METHODS) - 1)
    del host, bufd, hls
    return {"value": round(bytes_step / (ms / 1e3) / 1e9, 2), "unit": "GB/s", "h2d_bytes_per_step": int(world * h2d),
            "d2h_bytes_per_step": int(world * d2h), "ms_per_step": round(ms, 3), "steps": args.e2e_steps,
            "host_link_gbs": round(world * (h2d + d2h) / (ms / 1e3) / 1e9, 2),
            "counting": "value counts 8 m n bytes per call, as the device metric does: each X is copied from the host "
                        "once per step and factored by the three methods, so value = 3 x (X bytes) / time for the sweep; "
                        "host_link_gbs is the bytes actually moved over the host link per second",
            "one_copy_per_call": {"value": round(bytes_step / (ms_pc / 1e3) / 1e9, 2), "unit": "GB/s",
                                  "h2d_bytes_per_step": int(world * h2d_pc), "ms_per_step": round(ms_pc, 3),
                                  "steps": steps_pc,
                                  "note": "every call copies its X from pinned host memory (three copies of each X "
                                          "per step), reads its R back"},
            "note": "each X (and each [A b]) copied host->device once per step from pinned memory in pieces of "
                    "at most 1 GB (two at least) alternating over two copy streams into its own device buffer, so "
                    "copies overlap the factorisations still running (also the previous step's); every R and x "
                    "read back"}


# ------------------------------------------------------------------ shifted Cholesky-QR3


def _factor(q, meth, Xt, ws, arith):
    """R (host, float64) and status of one call in the given arithmetic."""
    prev = q.set_arith(arith)
    try:
        if meth == "tsqr":
            R, info = q.tsqr_qless(Xt, ws=ws)
        elif meth == "cholqr2":
            R, info = q.cholqr2_qless(Xt, ws=ws)
        else:
            R, _, info = q.svqb_qless(Xt, ws=ws)
        Rh, st = R.cpu().numpy(), info.cpu().tolist()
    finally:
        q.set_arith(prev)
    return Rh, st


def run_accuracy(q, lib, torch, dev, stream, Xs):
    """Is the default arithmetic FP64-class at full size?  Every sweep call (m = 2^25, n in
    NS, TSQR / Cholesky-QR2 / SVQB2) is made in the default arithmetic (double-float
    m-loops, FP64 n x n) and in native FP64 (every operation an FP64 instruction):
      * on the sweep's own X = G S (kappa 1e4): the relative difference of the two;
      * on X = H[:, J] H_64[:, K] R0 (signed sums of 64 random Walsh columns times a
        short-mantissa triangle, kappa(R0) ~ 1e4), exact in FP64 with R = sqrt(64 m) R0
        exactly: each arithmetic's error against that R, Frobenius and row-scaled, and their
        ratio.
    The native-FP64 arm is the same kernels' FP64 instantiation (plain FP64 sums), so the
    ratio answers "how far from what FP64 arithmetic gives in this design"."""
    import numpy as np

    from paper_2603_20889_gb300 import synth

    t0 = time.time()
    out = {"note": "default = double-float m-loops, FP64 n x n; f64 = native FP64 everywhere",
           "gauss": [], "exact": [],
           "exact_workload": "X = H[:, J] H_64[:, K] R0 (J, K random Walsh columns, 64 per entry; R0 = T1 diag(sigma) "
                             "T2 rounded to 2^-36, kappa(R0) ~ 1e4), m = 2^25, exact in FP64, R = sqrt(64 m) R0"}
    for n in NS:
        Xt = Xs[n].T
        ws = q.workspace(q.QL_AUTO, M, n, q.QL_F64, dev)
        for meth in METHODS:
            Rd, sd = _factor(q, meth, Xt, ws, q.QL_ARITH_DF)
            R6, s6 = _factor(q, meth, Xt, ws, q.QL_ARITH_F64)
            out["gauss"].append({"method": meth, "n": n, "df_vs_f64": rel_err(Rd, R6), "df_vs_f64_row": row_err(Rd, R6),
                                 "status": [sd, s6]})
        del ws
    worst = 0.0
    for n in NS:
        Xt_, R_ex = synth.hadamard_exact_device(M, n, KAPPA, seed=9000 + n, device=dev)
        Xt = Xt_.T
        ws = q.workspace(q.QL_AUTO, M, n, q.QL_F64, dev)
        for meth in METHODS:
            Rd, sd = _factor(q, meth, Xt, ws, q.QL_ARITH_DF)
            R6, s6 = _factor(q, meth, Xt, ws, q.QL_ARITH_F64)
            ed, e6 = rel_err(Rd, R_ex), rel_err(R6, R_ex)
            rd, r6 = row_err(Rd, R_ex), row_err(R6, R_ex)
            ratio = ed / max(e6, 1e-17)
            worst = max(worst, ratio)
            out["exact"].append({"method": meth, "n": n, "err_default": ed, "err_f64": e6, "ratio": round(ratio, 3),
                                 "row_err_default": rd, "row_err_f64": r6, "status": [sd, s6]})
        del Xt_, Xt, ws
        torch.cuda.empty_cache()
    out["max_ratio_default_over_f64"] = round(worst, 3)
    out["seconds"] = round(time.time() - t0, 1)
    return out


def run_scholqr3(q, lib, torch, dev, stream, reps=3):
    """Shifted Cholesky-QR3 on the condition sweep's kappa = 1e8 inputs (m = 2^25, beyond
    Cholesky-QR2's range): time per call, effective GB/s, the status of Cholesky-QR2 on the
    same X, and the relative difference of R from TSQR's."""
    from paper_2603_20889_gb300 import synth

    out = {"workload": "X = G S, m = 2^25, kappa = 1e8, FP64 storage", "calls": []}
    for n in (16, 64):
        X = synth.conditioned_device(M, n, 1e8, seed=2000 + n, device=dev)
        Xt = X.T
        ws = q.workspace(q.QL_AUTO, M, n, q.QL_F64, dev)
        R3, inf3 = q.scholqr3_qless(Xt, ws=ws)
        Rc, infc = q.cholqr2_qless(Xt, ws=ws)
        Rt, _ = q.tsqr_qless(Xt, ws=ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            q.scholqr3_qless(Xt, R3, inf3, ws)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        diff = float(torch.linalg.norm(R3 - Rt) / torch.linalg.norm(Rt))
        out["calls"].append({"n": n, "ms": round(ms, 3), "eff_gbs": round(8.0 * M * n / ms / 1e6, 1),
                             "status": inf3.tolist(), "cholqr2_status": infc.tolist(),
                             "rel_diff_vs_tsqr": diff, "tolerance_1e-13_n_kappa": 1e-13 * n * 1e8})
        del X, Xt, ws
        torch.cuda.empty_cache()
    return out


def run_kappa_rows(q, lib, torch, dev, stream, reps=2):
    """The condition sweep's other kappa values (1 and 1e8) at n = 16 and 64: time per call
    of TSQR, Cholesky-QR2 and SVQB2, their status, and the relative difference of each
    Gram method's R from TSQR's (held to 1e-13 n kappa only for kappa <= 1e6; at 1e8 the
    Gram methods square a condition number beyond 1 / sqrt(u) and may report breakdown)."""
    from paper_2603_20889_gb300 import synth

    out = {"workload": "X = G S, m = 2^25, kappa in {1, 1e8}, FP64 storage", "calls": []}
    for kappa in (1.0, 1e8):
        for n in (16, 64):
            X = synth.conditioned_device(M, n, kappa, seed=6000 + 2 * n + (1 if kappa > 1.0 else 0), device=dev)
            Xt = X.T
            ws = q.workspace(q.QL_AUTO, M, n, q.QL_F64, dev)
            Rt, it = q.tsqr_qless(Xt, ws=ws)
            Rc, ic = q.cholqr2_qless(Xt, ws=ws)
            Rs, _, iv = q.svqb_qless(Xt, ws=ws)
            calls = (("tsqr", lambda: q.tsqr_qless(Xt, Rt, it, ws)),
                     ("cholqr2", lambda: q.cholqr2_qless(Xt, Rc, ic, ws)),
                     ("svqb2", lambda: q.svqb_qless(Xt, Rs, info=iv, ws=ws)))
            row = {"kappa": kappa, "n": n}
            for name, fn in calls:
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    fn()
                e1.record(stream)
                torch.cuda.synchronize()
                row[name + "_ms"] = round(e0.elapsed_time(e1) / reps, 3)
            row["status"] = {"tsqr": it.tolist(), "cholqr2": ic.tolist(), "svqb2": iv.tolist()}
            for name, R in (("cholqr2", Rc), ("svqb2", Rs)):
                d = float(torch.linalg.norm(R - Rt) / torch.linalg.norm(Rt))
                row[name + "_rel_diff_vs_tsqr"] = d if math.isfinite(d) else None
            row["tolerance_1e-13_n_kappa"] = 1e-13 * n * kappa
            out["calls"].append(row)
            del X, Xt, ws, Rt, Rc, Rs
            torch.cuda.empty_cache()
    return out


def run_qform(q, lib, torch, dev, stream, reps=3):
    """Q = X R^{-1} for the sweep's shape (m = 2^25, kappa = 1e4) from TSQR's R: time per call,
    GB/s over the bytes moved (X read, Q written) and the orthogonality ||Q^T Q - I||_F."""
    from paper_2603_20889_gb300 import synth

    out = {"workload": "X = G S, m = 2^25, kappa = 1e4, FP64; R from TSQR", "calls": []}
    for n in (16, 64):
        X = synth.conditioned_device(M, n, KAPPA, seed=3000 + n, device=dev)
        Xt = X.T
        R, _ = q.tsqr_qless(Xt)
        Q, info = q.q_from_r(Xt, R)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            q.q_from_r(Xt, R, Q, info)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        orth = float(torch.linalg.norm(Q.T @ Q - torch.eye(n, dtype=torch.float64, device=dev)))
        out["calls"].append({"n": n, "ms": round(ms, 3), "gbs_moved": round(16.0 * M * n / ms / 1e6, 1),
                             "status": info.tolist(), "orthogonality": orth})
        del X, Xt, Q
        torch.cuda.empty_cache()
    return out


def run_project(q, lib, torch, dev, stream, reps=3):
    """Two-phase orthogonalisation of a block X (m = 2^25, n columns) against an orthonormal
    Y (k columns, Q of a Gaussian block): time per call, GB/s over the bytes moved (two passes
    read Y and the block twice and write the block twice), ||Y^T W||_F / ||X||_F."""
    from paper_2603_20889_gb300 import synth

    out = {"workload": "m = 2^25, Y = Q of a Gaussian m x k, X Gaussian m x n, FP64", "calls": []}
    for k, n in ((16, 16), (32, 32)):
        G = synth.conditioned_device(M, k, 1.0, seed=4000 + k, device=dev).T
        R, _ = q.tsqr_qless(G)
        Y, _ = q.q_from_r(G, R)
        X = synth.conditioned_device(M, n, 1.0, seed=4100 + n, device=dev).T
        W, C = q.project_out(Y, X)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            q.project_out(Y, X, W, C)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        orth = float(torch.linalg.norm(Y.T @ W) / torch.linalg.norm(X))
        moved = 8.0 * M * (2 * k + 2 * n) * 2
        out["calls"].append({"k": k, "n": n, "ms": round(ms, 3), "gbs_moved": round(moved / ms / 1e6, 1),
                             "rel_orthogonality": orth})
        del G, Y, X, W
        torch.cuda.empty_cache()
    return out


def run_wide(q, lib, torch, dev, stream, reps=2):
    """QR of wider X (m = 2^22, n = 128 and 256, kappa = 1e3, FP64) by 64-column panels:
    time per call, effective GB/s (8 m n bytes), ||Q^T Q - I||_F and the R difference from
    a one-panel check (TSQR R of the first 64 columns)."""
    from paper_2603_20889_gb300 import synth

    m = 1 << 22
    out = {"workload": "X = G S, m = 2^22, kappa = 1e3, FP64", "calls": []}
    for n in (128, 256):
        X = synth.conditioned_device(m, n, 1e3, seed=5000 + n, device=dev).T
        Q, R, info = q.qr_wide(X)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            q.qr_wide(X, R, Q, info)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        orth = float(torch.linalg.norm(Q.T @ Q - torch.eye(n, dtype=torch.float64, device=dev)))
        R1, _ = q.tsqr_qless(X[:, :64].contiguous().T.contiguous().T)
        d1 = float(torch.linalg.norm(R[:64, :64] - R1) / torch.linalg.norm(R1))
        out["calls"].append({"n": n, "ms": round(ms, 3), "eff_gbs": round(8.0 * m * n / ms / 1e6, 1),
                             "status": info.tolist(), "orthogonality": orth, "first_panel_vs_tsqr": d1})
        del X, Q, R
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ batched and serving forms


def run_batched(q, lib, torch, dev, stream, count=512):
    """Uneven batch (m log-uniform in [2^10, 2^20], n in {4..48}, kappa log-uniform in
    [1, 1e6], FP64), the method of each problem chosen by the library (method_hint = QL_AUTO
    with the construction kappa as kappa_hint): the batched form (its persistent launches,
    plain and CUDA-graph replay) against a loop of one single call per matrix with the same
    method on the same stream, and against the all-TSQR batch.  Accuracy: sampled instances
    against the single-call results and the smallest against LAPACK's QR on the host."""
    import ctypes

    import numpy as np

    from paper_2603_20889_gb300 import synth

    insts = synth.batched_instances(count)
    Xs, outs = [], []
    for it in insts:
        Xt = synth.conditioned_device(it.m, it.n, it.kappa, it.seed, device=dev)
        R = torch.empty((it.n, it.n), dtype=torch.float64, device=dev)
        info = torch.zeros(2, dtype=torch.int32, device=dev)
        Xs.append(Xt)
        outs.append((R, info))

    def plan(hint):
        probs = [q.Problem(m=it.m, n=it.n, ld=it.m, X=Xt.data_ptr(), dtype=q.QL_F64, kind=0, b=None,
                           R=R.data_ptr(), x=None, info=info.data_ptr(), method_hint=hint, kappa_hint=it.kappa)
                 for it, Xt, (R, info) in zip(insts, Xs, outs)]
        arr = (q.Problem * count)(*probs)
        nb = lib.ql_batch_workspace_bytes(count, arr)
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        assert lib.ql_batch_prepare(count, arr, ws.data_ptr(), nb, q._stream_ptr(stream)) == 0
        meth = (ctypes.c_int32 * count)()
        assert lib.ql_batch_methods(ws.data_ptr(), meth, count) == 0
        return ws, list(meth)

    sptr = q._stream_ptr(stream)
    total_bytes = sum(8.0 * it.m * it.n for it in insts)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ws_t, _ = plan(q.QL_TSQR)
    ms_tsqr = timed(lambda: lib.ql_batch_launch(ws_t.data_ptr(), sptr), 5)
    del ws_t
    ws, methods = plan(q.QL_AUTO)
    ms_batch = timed(lambda: lib.ql_batch_launch(ws.data_ptr(), sptr), 5)
    side = torch.cuda.Stream(device=dev)  # capture needs a non-default stream
    side.wait_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        lib.ql_batch_launch(ws.data_ptr(), q._stream_ptr(side))
    stream.wait_stream(side)
    ms_graph = timed(g.replay, 5)
    Rb = [o[0].clone() for o in outs]
    bad = [i for i, o in enumerate(outs) if o[1].cpu().tolist() != [0, 0]]
    wsl = torch.empty(lib.ql_workspace_bytes(q.QL_AUTO, 1 << 20, 48, q.QL_F64), dtype=torch.uint8, device=dev)

    def loop():  # the same method per matrix, one single call each
        for it, Xt, (R, info), mth in zip(insts, Xs, outs, methods):
            fn = lib.ql_cholqr2_qless if mth == q.QL_CHOLQR2 else lib.ql_tsqr_qless
            fn(it.m, it.n, Xt.data_ptr(), q.QL_F64, it.m, R.data_ptr(), it.n, info.data_ptr(), wsl.data_ptr(),
               wsl.numel(), sptr)

    ms_loop = timed(loop, 2)
    # batched vs single-call parity on a sample, and the smallest instances against LAPACK's
    # Householder QR on the host (the parity against the oracle is the tests' job)
    worst = 0.0
    for i in range(0, count, 16):
        it = insts[i]
        e = float((Rb[i] - outs[i][0]).norm() / outs[i][0].norm())
        worst = max(worst, e / tolerance(it.n, max(it.kappa, 10.0)))
    small = sorted(range(count), key=lambda i: insts[i].m * insts[i].n)[:4]
    worst_lapack = 0.0
    for i in small:
        it = insts[i]
        Xh = Xs[i].double().cpu().numpy().T
        Rh = Rb[i].cpu().numpy().T  # stored column-major
        worst_lapack = max(worst_lapack, rel_err(Rh, lapack_r(Xh)) / tolerance(it.n, max(it.kappa, 10.0)))
    n_gram = sum(1 for m in methods if m == q.QL_CHOLQR2)
    del Xs
    return {
        "workload": f"{count} uneven FP64 problems: m log-uniform in [2^10, 2^20], n in {{4..48}}, "
                    "kappa log-uniform in [1, 1e6]",
        "method": "per problem (method_hint = QL_AUTO, kappa_hint = construction kappa): TSQR problems in one "
                  "persistent launch, Cholesky-QR2 problems in grouped persistent Gram launches per column class "
                  "and pass, gated FP64 TSQR redo launch",
        "methods_chosen": {"tsqr": count - n_gram, "cholqr2": n_gram},
        "methods_per_instance": "".join("C" if m == q.QL_CHOLQR2 else "T" for m in methods),
        "solves_per_s_batched": round(count / (ms_batch / 1e3), 1),
        "solves_per_s_graph": round(count / (ms_graph / 1e3), 1),
        "solves_per_s_loop": round(count / (ms_loop / 1e3), 1),
        "solves_per_s_batched_all_tsqr": round(count / (ms_tsqr / 1e3), 1),
        "speedup_vs_loop": round(ms_loop / ms_graph, 2),
        "ms_batched": round(ms_batch, 3), "ms_graph": round(ms_graph, 3), "ms_loop": round(ms_loop, 3),
        "ms_batched_all_tsqr": round(ms_tsqr, 3),
        "eff_gbs_batched": round(total_bytes / (ms_graph / 1e3) / 1e9, 1),
        "eff_gbs_loop": round(total_bytes / (ms_loop / 1e3) / 1e9, 1),
        "status_errors": len(bad), "max_err_over_tol_vs_single": round(worst, 4),
        "max_err_over_tol_vs_lapack": round(worst_lapack, 4),
    }


def run_serving(q, lib, torch, dev, count=20000, rate=2000.0, budget=60 * 10 ** 9, max_wall=60.0):
    """Poisson stream of Q-less QR / least-squares requests through the continuous-batching
    server.  Payloads are views of device-resident pools (one 2^22 x 65 matrix per kappa
    bucket, FP64 and FP32 copies), so no host->device copy happens after arrival."""
    import numpy as np

    from paper_2603_20889_gb300 import synth

    reqs = synth.serving_stream(count, rate)
    kb = [1.0, 1e2, 1e4, 1e6]
    M = 1 << 22
    pools64 = [synth.conditioned_device(M, 65, k, seed=77 + i, device=dev) for i, k in enumerate(kb)]
    pools32 = [p.float() for p in pools64]
    # the server's streams do not wait on the default stream: the pools must be complete
    torch.cuda.synchronize()
    srv = q.Server(budget, 8192, 4)
    t0 = time.perf_counter()
    tickets = []
    submitted = 0
    for r in reqs:
        now = time.perf_counter() - t0
        if now > max_wall:
            break
        if r.arrival_s > now:
            time.sleep(r.arrival_s - now)
        b = min(range(4), key=lambda i: abs(math.log10(kb[i]) - math.log10(r.kappa)))
        pool = pools64[b] if r.dtype == "f64" else pools32[b]
        base = pool.data_ptr()
        el = 8 if r.dtype == "f64" else 4
        req = q.Request(m=r.m, n=r.n, ld=M, X=base, dtype=q.QL_F64 if r.dtype == "f64" else q.QL_F32,
                        kind=1 if r.kind == "lstsq" else 0,
                        b=base + 64 * M * el if r.kind == "lstsq" else None, kappa_hint=r.kappa,
                        method_hint=q.QL_AUTO)
        tickets.append((srv.submit(req), r, b))
        submitted += 1
    t_sub = time.perf_counter() - t0
    srv.drain(max(1.0, max_wall - t_sub))
    t_all = time.perf_counter() - t0
    st = srv.stats()
    # alone-vs-mix check on a sample: the served R against a single TSQR call
    worst = 0.0
    bad = 0
    codes = []
    cudart = lib
    for tk, r, b in tickets[:: max(1, len(tickets) // 24)]:
        s, res = srv.poll(tk)
        if s != 0 or res.status != 0:
            bad += 1
            codes.append({"poll": int(s), "status": int(res.status), "m": r.m, "n": r.n, "kind": r.kind,
                          "dtype": r.dtype, "kappa": r.kappa})
            continue
        n1 = r.n + 1 if r.kind == "lstsq" else r.n
        buf = np.zeros(n1 * n1)
        cudart.cudaMemcpy(ctypes.c_void_p(buf.ctypes.data), ctypes.c_void_p(res.R), ctypes.c_size_t(n1 * n1 * 8),
                          ctypes.c_int(2))
        Rs = buf.reshape((n1, n1), order="F")
        pool = pools64[b] if r.dtype == "f64" else pools32[b]
        if r.kind == "lstsq":  # [A b] with b = pool column 64
            X = torch.cat([pool[:r.n, :r.m], pool[64:65, :r.m]]).contiguous().T
        else:
            X = pool[:r.n, :r.m].T
        Ra, _ = q.tsqr_qless(X)
        Ra = Ra.cpu().numpy()
        worst = max(worst, rel_err(Rs, Ra) / tolerance(n1, max(r.kappa, 10.0)))
    srv.close()
    # the same request list as one plain call per request, back to back on one stream (the
    # method the batch plan would pick: Cholesky-QR2 from 24 columns at kappa <= 1e6)
    nloop = min(len(tickets), 2000)
    wsl = torch.empty(lib.ql_workspace_bytes(q.QL_AUTO, M, 64, q.QL_F64), dtype=torch.uint8, device=dev)
    Rl = torch.empty(65 * 65, dtype=torch.float64, device=dev)
    xl = torch.empty(66, dtype=torch.float64, device=dev)
    infl = torch.zeros(2, dtype=torch.int32, device=dev)
    sp = q._stream_ptr(torch.cuda.current_stream())

    def one(r, b):
        pool = pools64[b] if r.dtype == "f64" else pools32[b]
        dt = q.QL_F64 if r.dtype == "f64" else q.QL_F32
        el = 8 if r.dtype == "f64" else 4
        ncols = r.n + (1 if r.kind == "lstsq" else 0)
        meth = q.QL_CHOLQR2 if (ncols >= 24 and r.kappa <= 1e6) else q.QL_TSQR
        if r.kind == "lstsq":
            lib.ql_lstsq_qless(r.m, r.n, pool.data_ptr(), M, pool.data_ptr() + 64 * M * el, dt, meth, xl.data_ptr(),
                               xl[r.n:].data_ptr(), None, infl.data_ptr(), wsl.data_ptr(), wsl.numel(), sp)
        elif meth == q.QL_CHOLQR2:
            lib.ql_cholqr2_qless(r.m, r.n, pool.data_ptr(), dt, M, Rl.data_ptr(), r.n, infl.data_ptr(), wsl.data_ptr(),
                                 wsl.numel(), sp)
        else:
            lib.ql_tsqr_qless(r.m, r.n, pool.data_ptr(), dt, M, Rl.data_ptr(), r.n, infl.data_ptr(), wsl.data_ptr(),
                              wsl.numel(), sp)

    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for tk, r, b in tickets[:nloop]:
        one(r, b)
    e1.record()
    torch.cuda.synchronize()
    loop_sps = nloop / (e0.elapsed_time(e1) / 1e3)
    del pools64, pools32
    return {
        "workload": f"Poisson {rate:.0f} req/s, m log-uniform in [2^12, 2^22], n in {{2..64}}, 30% FP32, "
                    "20% least squares, kappa log-uniform in [1, 1e6] (kappa_hint, method_hint = QL_AUTO), "
                    f"{budget / 1e9:.0f} GB budget",
        "loop_solves_per_s": round(loop_sps, 1),
        "loop": f"the first {nloop} requests as one plain call each, back to back, same methods",
        "submitted": submitted, "completed": int(st.completed), "offered_s": round(t_sub, 2),
        "wall_s": round(t_all, 2), "solves_per_s": round(st.completed / max(t_all, 1e-9), 1),
        "p50_ms": round(st.p50_ms, 3), "p99_ms": round(st.p99_ms, 3), "mean_ms": round(st.mean_ms, 3),
        "hbm_budget_gb": round(budget / 1e9, 2), "hbm_peak_gb": round(st.hbm_peak_bytes / 1e9, 2), "sample_status_errors": bad, "sample_failures": codes,
        "max_err_over_tol_alone_vs_mix": round(worst, 4),
    }


# ------------------------------------------------------------------ the oracle on the host


def oracle_sample(seconds: float):
    """Time the CPU oracle (plain Householder, long-double accumulation, one thread) on a
    bounded row sample of the same sweep; returns (GB/s in the metric's unit, detail)."""
    import numpy as np

    import oracle
    from paper_2603_20889_gb300 import synth

    # calibrate: rows per second at n = 8
    Xc = synth.conditioned(20000, 8, KAPPA, seed=7)
    t0 = time.perf_counter()
    oracle.householder_r(Xc)
    dt = max(time.perf_counter() - t0, 1e-4)
    flop_rate = 2.0 * 20000 * 64 / dt  # oracle Householder flops per second
    budget = seconds / (len(NS) * len(METHODS))
    total_bytes, total_s, parts = 0.0, 0.0, []
    for n in NS:
        ms_rows = int(max(256, min(M, budget * flop_rate / (2.0 * n * n))))
        X = synth.conditioned(ms_rows, n, KAPPA, seed=1000 + n)
        for meth in METHODS:
            t0 = time.perf_counter()
            if meth == "tsqr":
                oracle.householder_r(X)
            elif meth == "cholqr2":
                oracle.cholqr2(X)
            else:
                oracle.svqb2(X)
            s = time.perf_counter() - t0
            total_s += s
            total_bytes += 8.0 * ms_rows * n
            parts.append(f"{meth} n={n} m={ms_rows}")
    # least squares through the QR of [A b] (FP64- and FP32-stored A; the oracle computes in
    # FP64 on the stored values, the bytes are those of the stored [A b])
    ms_rows = int(max(256, min(LS_M, budget * flop_rate / (2.0 * (LS_N + 1) ** 2))))
    A, b, _ = synth.lstsq_case(ms_rows, LS_N, 1e3, seed=4242)
    for name, itemsize in (("lstsq_f64", 8.0), ("lstsq_f32", 4.0)):
        Ai, bi = (A, b) if itemsize == 8.0 else (A.astype(np.float32), b.astype(np.float32))
        t0 = time.perf_counter()
        oracle.lstsq(Ai, bi)
        s = time.perf_counter() - t0
        total_s += s
        total_bytes += itemsize * ms_rows * (LS_N + 1)
        parts.append(f"{name} n={LS_N} m={ms_rows}")
    return total_bytes / total_s / 1e9, total_s, "; ".join(parts)


def cpu_context(rows: int = 1 << 22):
    """All host cores, LAPACK's Householder QR through torch.linalg.qr(mode='r') on a row
    sample of every sweep width: a context number beside the single-thread oracle (a
    baseline, not the target)."""
    import torch

    from paper_2603_20889_gb300 import synth

    total_bytes, total_s, parts = 0.0, 0.0, []
    for n in NS:
        X = torch.from_numpy(synth.conditioned(rows, n, KAPPA, seed=1000 + n))
        torch.linalg.qr(X[: 1 << 12], mode="r")  # warm-up
        t0 = time.perf_counter()
        torch.linalg.qr(X, mode="r")
        s = time.perf_counter() - t0
        total_s += s
        total_bytes += 8.0 * rows * n
        parts.append(f"n={n}: {s * 1e3:.1f} ms")
        del X
    return {"value": round(total_bytes / total_s / 1e9, 3), "unit": "GB/s", "cores": torch.get_num_threads(),
            "kind": "torch.linalg.qr(mode='r') (LAPACK Householder), one call per n",
            "sample": f"m = {rows} rows of the sweep's X for n in {NS} (TSQR-equivalent: one R per X); " + "; ".join(parts)}


def cpu_baseline(seconds):
    v, s, sample = oracle_sample(seconds)
    return {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"row samples of the same sweep ({s:.1f} s of CPU): {sample}"}


# ------------------------------------------------------------------ one call shape


def run_case(spec: str, reps: int = 3) -> dict:
    """One call shape of the sweep (METHOD:N:M), run reps times after one warm-up call:
    the small, self-contained program that kernel profiles are taken on."""
    import torch

    import paper_2603_20889_gb300 as q
    from paper_2603_20889_gb300 import synth

    method, n, m = spec.split(":")
    n, m = int(n), int(m)
    q.load_library()
    X = synth.conditioned_device(m, n, KAPPA, seed=n).T
    ws = q.workspace(q.QL_AUTO, m, n, q.QL_F64)
    R = torch.empty((n, n), dtype=torch.float64, device="cuda").T
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    call = {"tsqr": lambda: q.tsqr_qless(X, R, info, ws), "cholqr2": lambda: q.cholqr2_qless(X, R, info, ws),
            "svqb2": lambda: q.svqb_qless(X, R, None, 0.0, info, ws)}[method]
    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"case": spec, "ms": round(ms, 3), "eff_gbs": round(8 * m * n / ms / 1e6, 1), "info": info.tolist()}


# ------------------------------------------------------------------ main


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.case:
        print(json.dumps(run_case(args.case)))
        return 0
    if args.impl == "reference":
        if rank != 0:
            return 0
        per_step = []
        for _ in range(args.warmup):
            oracle_sample(min(args.cpu_seconds, 4.0) / 4)
        for _ in range(args.steps):
            v, s, sample = oracle_sample(args.cpu_seconds / max(args.steps, 1))
            per_step.append((v, s))
        value = statistics.median(v for v, _ in per_step)
        ms = statistics.mean(s for _, s in per_step) * 1e3
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "bounded row samples per step (the oracle is a CPU program)"},
            "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return 0
    if world > 1:
        import torch

        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        if args.cpu_context:
            try:
                out["cpu_context"] = cpu_context()
            except Exception as exc:
                out["cpu_context"] = {"error": repr(exc)[:300]}
        print(json.dumps(out))
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
