"""Benchmark: element matrices per second of batched element-local assembly.

Workload (one step = one pass of the whole hot path over one batch): the
Helmholtz form  int grad u . grad v + f u v  with P2 test/trial functions and
a P2 coefficient f, on 1,000,000 random affine tetrahedra (collapsed
Gauss-Jacobi 4^3 = 64-point rule, 10 x 10 FP64 element matrices), inputs
resident in HBM.  Each step is one launch of the flop-reduced kernel chosen by
the planner (pre-evaluated reference tensors, FP32 contraction, FP64
geometry).

Also reported: the plain FP64 GPU kernel (the comparator) on the same
workload, the end-to-end rate through the host-buffer C ABI call (copies
inside the timed region), the roofline of the dominant kernel against the
measured HBM bandwidth, clocks during the timed region, and the FP64 CPU
oracle on a bounded sample of the workload (rank 0, N = 1).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "helmholtz_p2_1M", "form": "helmholtz", "degree": 2, "elements": 1_000_000,
            "quad_points": 64, "local_matrix": "10x10 f64"}
METRIC = "element matrices/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# committed ncu summaries of the timed kernels: profile file and the sources its kernel is built from
PROFILES = {
    "helmholtz_p2_1M": ("helmholtz_p2_pre_1M.md", ["common.cuh", "layout.h", "pre_stream.cuh", "planner.cpp"]),
    "elasticity_p3_200k": ("elasticity_p3_pre_stream_200k.md",
                           ["common.cuh", "layout.h", "pre_stream.cuh", "stream_batched.cuh", "pre_vec_stream.cuh",
                            "pre_vec.cuh", "sym.cuh", "planner.cpp"]),
    "neohookean_p2_500k": ("neohookean_p2_se_500k.md",
                           ["common.cuh", "layout.h", "launch.cuh", "se_vec.cuh", "sym.cuh", "log_f64.cuh",
                            "log_table.h", "planner.cpp"]),
    "neohookean_p2_500k@bf16x2": ("neohookean_p2_tc_500k.md",
                                  ["common.cuh", "layout.h", "launch.cuh", "mbar.cuh", "tc.cuh", "nh_tc.cuh",
                                   "log_f64.cuh", "log_table.h", "kernels_tc.cu"]),
    "neohookean_p3_100k@bf16x2": ("neohookean_p3_tc_100k.md",
                                  ["common.cuh", "layout.h", "launch.cuh", "mbar.cuh", "tc.cuh", "nh_tce.cuh",
                                   "log_f64.cuh", "log_table.h", "kernels_tc.cu"]),
    "helmholtz_p2_global_1M": ("global_helmholtz_p2_1M.md",
                               ["common.cuh", "layout.h", "kernels.h", "pre_stream.cuh", "pre_combine.cuh", "planner.cpp"]),
    "helmholtz_load_p2_1M": ("helmholtz_load_p2_1M.md", ["common.cuh", "layout.h", "pre_stream.cuh"]),
    "neohookean_residual_p2_500k": ("neohookean_residual_p2_500k.md",
                                    ["common.cuh", "layout.h", "launch.cuh", "vec_forms.cuh", "log_f64.cuh",
                                     "log_table.h"]),
}


def kernel_source_hash(names):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1604_05872_gb300", "csrc")
    for name in names:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload):
    """DRAM bytes per launch of the workload's timed kernel from its committed ncu
    summary, or None when there is none or the kernel sources changed since."""
    if workload not in PROFILES:
        return None
    name, sources = PROFILES[workload]
    try:
        txt = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    s = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    if not m or not s or s.group(1) != kernel_source_hash(sources):
        return None
    return float(m.group(1))


CLOCKS_LOG = None  # --clocks-log: path of an nvidia-smi log of the timed regions


class ClockSampler:
    """SM clock and clock-event reasons sampled through NVML (libnvidia-ml,
    read-only queries) by a background thread during the timed region, plus,
    with --clocks-log, an nvidia-smi log of the same quantities."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index, period=0.002):
        self.index, self.period = index, period
        self.samples, self.max_mhz = [], None
        self.nvml = None
        self.proc = None

    def _init_nvml(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return False
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
                return False
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx)) == 0:
                self.max_mhz = mx.value
            self.nvml, self.h = lib, h
            return True
        except OSError:
            return False

    def _run(self):
        import ctypes
        mhz, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        get_r = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nvml.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop.is_set():
            if self.nvml.nvmlDeviceGetClockInfo(self.h, ctypes.c_int(1), ctypes.byref(mhz)) == 0:
                r = rs.value if get_r(self.h, ctypes.byref(rs)) == 0 else 0
                self.samples.append((mhz.value, r))
            time.sleep(self.period)

    def __enter__(self):
        import threading
        try:
            if not CLOCKS_LOG:
                raise OSError("no nvidia-smi log requested")
            d = os.path.dirname(os.path.abspath(CLOCKS_LOG))
            os.makedirs(d, exist_ok=True)
            self.log = open(CLOCKS_LOG, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv", "-lms", "200"], stdout=self.log, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.stop = threading.Event()
        if self._init_nvml():
            self.thread = threading.Thread(target=self._run, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.samples and time.time() - t0 < 2.0:
                time.sleep(0.001)
            self.samples.clear()
        else:
            self.thread = None
        return self

    def __exit__(self, *a):
        self.stop.set()
        if self.thread:
            self.thread.join(timeout=2)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.log.close()

    def summary(self):
        if not self.samples:
            return None
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": float(np.median([m for m, _ in self.samples])), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(self.samples), "source": "nvml"}


def make_inputs(E, seed_offset=0):
    from paper_1604_05872_gb300 import inputs
    coords, f = inputs.workload(inputs.HELMHOLTZ, 2, E, seed=inputs.SEED + seed_offset)
    return coords, f


def cpu_baseline(form, p, coords, coeffs, budget_s=15.0):
    """FP64 oracle on a bounded sample of the workload (host cores, OpenMP over elements)."""
    import oracle
    threads = max(1, os.cpu_count() or 1)
    n = 200
    t0 = time.perf_counter()
    oracle.assemble(form, p, coords[:n], None if coeffs is None else coeffs[:n], nthreads=threads)
    dt = time.perf_counter() - t0
    n2 = int(min(len(coords), max(n, n * budget_s / max(dt, 1e-4) * 0.8)))
    t0 = time.perf_counter()
    oracle.assemble(form, p, coords[:n2], None if coeffs is None else coeffs[:n2], nthreads=threads)
    dt = time.perf_counter() - t0
    return {"value": n2 / dt, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": "first %d elements of the workload, FP64 quadrature-mode loop nest, %.1f s" % (n2, dt)}


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle as it stands, on host cores."""
    if rank != 0:
        return
    coords, f = make_inputs(20000)
    import oracle
    threads = max(1, os.cpu_count() or 1)
    per = 2000
    for _ in range(args.warmup):
        oracle.assemble(1, 2, coords[:per], f[:per], nthreads=threads)
    t0 = time.perf_counter()
    for k in range(args.steps):
        s = (k * per) % (len(coords) - per)
        oracle.assemble(1, 2, coords[s:s + per], f[s:s + per], nthreads=threads)
    dt = time.perf_counter() - t0
    value = args.steps * per / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, sample_per_step=per),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle",
                             "sample": "%d elements of the workload per step" % per},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


WORKLOADS = {
    # name: (form, degree, elements, anisotropic)
    "helmholtz_p2_1M": (1, 2, 1_000_000, False),
    "mass_p1_10k": (0, 1, 10_000, False),
    "elasticity_p3_200k": (2, 3, 200_000, True),
    "neohookean_p2_500k": (3, 2, 500_000, False),
    "neohookean_p3_100k": (3, 3, 100_000, False),
}
L2_BYTES = 129_000_000                                # GB300 L2 (129 MB)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x 2 flops x max clock
FP64_PEAK_TINSTR = 152 * 2 * 2.07e9 / 1e12          # SMs x FP64 lanes per clock x max clock (lane-instructions)


def fp64_ops_per_element(form, p, variant, Q):
    """FP64 lane-instructions per element of the flop-reduced kernels: 30 for
    the geometry (9 subtractions for J, 18 for the adjugate's 2x2 minors, 3 for
    det J), plus NEO_POINT_FP64 per Neo-Hookean point."""
    return 30 + (NEO_POINT_FP64 * Q if form == 3 else 0)


# FP64 lane-instructions per Neo-Hookean point: F = I + grad u (3 additions), the
# cofactors of F (18) and det F (3), two tests of det F, and ln det F by the
# table-driven logarithm (13); the tensor-core kernel tests det F with integer ops
NEO_POINT_FP64 = 3 + 18 + 3 + 2 + 13
NEO_POINT_FP64_TC = 3 + 18 + 3 + 13


def precision_of(args, fea, form, p):
    """(precision code, name, uses the tensor-core kernel) for a (form, degree)."""
    names = {"fp32": fea.PREC_FP32, "bf16x2": fea.PREC_BF16X2, "fp64": fea.PREC_FP64}
    f32 = bool(args.out_f32)  # a tensor-core kernel exists where the split-BF16 plan differs from the FP32 one
    tc = fea.plan(form, p, precision=fea.PREC_BF16X2, out_f32=f32) != fea.plan(form, p, precision=fea.PREC_FP32, out_f32=f32)
    if args.precision == "auto":  # the tensor cores wherever the split-BF16 plan has a kernel for them
        return (fea.PREC_BF16X2, "bf16x2", True) if tc else (fea.PREC_FP32, "fp32", False)
    prec = names[args.precision]
    return prec, args.precision, tc and prec == fea.PREC_BF16X2


def tc_flops_per_element(form, p):
    """Useful tensor-core flops per element of the split-BF16 Neo-Hookean kernels,
    2 flops per MAC.  P2 (reference tables as the shared operand): rows = 2 x the
    symmetric basis pairs (hi and lo parts), 9 columns (c, d) per element,
    K = 9 (Q + 1) (the points and the point-summed term), two passes (hi and lo
    parts of H).  P3 (one product per element): the 3 n_s x 3 n_s blocks S and T
    over the Q points, three split chains (hi hi, hi lo, lo hi).  Mass and Helmholtz
    (FP32 output): the pre-evaluated contraction, r terms x n_s^2 entries, four split
    products."""
    ns = (p + 1) * (p + 2) * (p + 3) // 6
    Q = (p + 1) ** 3
    if form in (0, 1):  # pre-evaluated scalar forms: [elements x r] x [r x n^2], four split products
        r = 1 if form == 0 else 6 + ns
        return 2 * 4 * r * ns * ns
    if p == 2:
        return 2 * 2 * (ns * (ns + 1)) * 9 * 9 * (Q + 1)
    return 2 * 3 * 2 * (3 * ns) ** 2 * Q


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="helmholtz_p2_1M",
                    choices=sorted(WORKLOADS) + sorted(VECTOR_WORKLOADS) + ["stream_64req_2M", "helmholtz_p2_global_1M",
                                                                            "helmholtz_bernstein_p4_200k"])
    ap.add_argument("--elements", type=int, default=0, help="override the element count")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--tuning", default=os.path.join(ROOT, "paper_1604_05872_gb300", "data", "tuning_gb300.json"),
                    help="tuning JSON (records + MLP) for the stream workload ('' for the flop-count choice only)")
    ap.add_argument("--out-f32", action="store_true", help="FP32 output (element matrices stored as float)")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16x2", "fp64"],
                    help="contraction arithmetic; auto = split-BF16 tensor cores where a tensor-core kernel exists "
                         "(Neo-Hookean P2), FP32 elsewhere")
    ap.add_argument("--clocks-log", default="", help="also log nvidia-smi clocks of the timed regions to this CSV")
    args = ap.parse_args()
    global CLOCKS_LOG
    CLOCKS_LOG = args.clocks_log or None
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    import paper_1604_05872_gb300 as fea

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    fea.load()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    if args.workload == "stream_64req_2M":
        line = run_stream(args, fea, torch, barrier, max_over_ranks, world, local)
    elif args.workload in VECTOR_WORKLOADS:
        line = run_vector(args, fea, torch, barrier, max_over_ranks, world, rank, local)
    elif args.workload == "helmholtz_p2_global_1M":
        line = run_global(args, fea, torch, barrier, max_over_ranks, world, rank, local)
    elif args.workload == "helmholtz_bernstein_p4_200k":
        line = run_bernstein(args, fea, torch, barrier, max_over_ranks, world, rank, local)
    else:
        line = run_single(args, fea, torch, barrier, max_over_ranks, world, rank, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_single(args, fea, torch, barrier, max_over_ranks, world, rank, local):
    from paper_1604_05872_gb300 import inputs
    form, p, E0, aniso = WORKLOADS[args.workload]
    E = args.elements or E0
    coords, coeffs = inputs.workload(form, p, E, seed=inputs.SEED + rank, anisotropic=aniso)  # own shard per rank
    c = torch.from_numpy(coords).cuda()
    fc = None if form == 0 else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    f32 = bool(args.out_f32)
    out = fea.empty_out(form, p, E, out_f32=f32)
    n = out.shape[1]
    esz = 4 if f32 else 8
    stream = torch.cuda.current_stream()
    prec, prec_name, tc = precision_of(args, fea, form, p)
    pl = fea.plan(form, p, precision=prec, out_f32=f32)
    bytes_elem = 96 + 8 * fea.coeff_len(form, p) + esz * n * n

    for _ in range(args.warmup):
        fea.assemble(form, p, c, fc, out=out, out_f32=f32, precision=prec)
    fea.sync()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    small = E * bytes_elem <= L2_BYTES
    if not small:
        # inputs and outputs larger than L2: back-to-back steps, one pair of events
        with ClockSampler(local) as clk:
            ev0.record(stream)
            for _ in range(args.steps):
                fea.assemble(form, p, c, fc, out=out, out_f32=f32, precision=prec)
            ev1.record(stream)
            barrier()
        ms = ev0.elapsed_time(ev1) / args.steps
    else:
        # a step that fits L2: flush it (a write larger than L2) before every step and time each step
        # with its own events; the flush also keeps the device busy while the host issues the launch
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with ClockSampler(local) as clk:
            for a, b in evs:
                flush.fill_(1.0)
                a.record(stream)
                fea.assemble(form, p, c, fc, out=out, out_f32=f32, precision=prec)
                b.record(stream)
            torch.cuda.synchronize()
            barrier()
        ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
        del flush
    fea.sync()
    ms_max = max_over_ranks(ms)
    value = E * world / (ms_max * 1e-3)

    # plain FP64 comparator on the same workload (a bounded prefix of it for the slowest forms)
    En = int(min(E, max(1000, 0.5e12 / pl["flops_naive"])))
    out64 = out if not f32 else fea.empty_out(form, p, En)
    fea.assemble(form, p, c[:En], fc, out=out64[:En], precision=fea.PREC_FP64, variant=fea.VARIANT_NAIVE)
    barrier()
    nsteps = 2
    ev0.record(stream)
    for _ in range(nsteps):
        fea.assemble(form, p, c[:En], fc, out=out64[:En], precision=fea.PREC_FP64, variant=fea.VARIANT_NAIVE)
    ev1.record(stream)
    barrier()
    ms_naive = ev0.elapsed_time(ev1) / nsteps
    fea.sync()
    naive_rate = En / (ms_naive * 1e-3)

    # end to end through the host-buffer C ABI call (copies inside the timed region)
    hc = torch.from_numpy(coords).pin_memory()
    hf = None if fc is None else fc.cpu().pin_memory()
    del out64
    ho = torch.empty((E, n, n), dtype=torch.float32 if f32 else torch.float64).pin_memory()
    for _ in range(2):
        fea.assemble_host(form, p, hc, hf, ho, out_f32=f32, precision=prec)
    barrier()
    e2e_steps = max(3, args.steps // 4)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        fea.assemble_host(form, p, hc, hf, ho, out_f32=f32, precision=prec)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) / e2e_steps * 1e3)

    hbm, peak_kind = peaks()
    alg_bytes = E * bytes_elem
    flops = E * (tc_flops_per_element(form, p) if tc else pl["flops_run"])
    f64 = E * (30 + NEO_POINT_FP64_TC * pl["quad_points"] if tc and form == 3
               else fp64_ops_per_element(form, p, pl["variant"], pl["quad_points"]))
    t_hbm = alg_bytes / (hbm * 1e9)
    bf16, bf16_kind = bf16_peak()
    t_f32 = flops / ((bf16 if tc else FP32_PEAK_TFLOPS) * 1e12)
    t_f64 = f64 / (FP64_PEAK_TINSTR * 1e12)
    if t_hbm >= max(t_f32, t_f64):
        roof = {"bound": "hbm", "achieved": alg_bytes / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_kind": peak_kind}
    elif t_f32 >= t_f64 and tc:
        roof = {"bound": "tensor", "achieved": flops / (ms * 1e-3) / 1e12, "peak": bf16, "unit": "TFLOP/s",
                "peak_kind": bf16_kind + " bf16 dense (split-BF16 products)"}
    elif t_f32 >= t_f64:
        roof = {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "peak_kind": "derived: FP32 lanes x clock"}
    else:
        roof = {"bound": "alu", "achieved": f64 / (ms * 1e-3) / 1e12, "peak": FP64_PEAK_TINSTR,
                "unit": "T FP64 lane-instructions/s", "peak_kind": "derived: FP64 lanes x clock"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = profiled_traffic(args.workload + ("@bf16x2" if tc else "")) if E == E0 and not f32 else None
    roof["alg_bytes_per_launch"] = alg_bytes
    roof["bound_times_ms"] = {"hbm": t_hbm * 1e3, ("tensor" if tc else "fp32"): t_f32 * 1e3, "fp64": t_f64 * 1e3}
    if tc:
        roof["tensor_achieved_tflops"] = flops / (ms * 1e-3) / 1e12
        roof["tensor_frac"] = roof["tensor_achieved_tflops"] / bf16
    cfg = {"workload": args.workload, "form": ["mass", "helmholtz", "elasticity", "neohookean"][form],
           "degree": p, "elements": E, "quad_points": pl["quad_points"], "local_matrix": "%dx%d %s" % (n, n, "f32" if f32 else "f64"),
           "variant": fea.VARIANT_NAMES[pl["variant"]] + ((" (per-point pre-evaluation on tcgen05)" if p == 2 else
                                                          " (one S, T product per element on tcgen05)") if tc else ""),
           "tile": pl["tile"], "geometry": "f64",
           "contraction": "bf16x2 split operands on tcgen05 tensor cores, f32 accumulation" if tc else prec_name,
           "parallelism": "dp%d (element shards)" % world,
           "l2": "inputs+outputs %.0f MB per step%s" % (alg_bytes / 1e6, " > 129 MB L2; no flush" if not small
                                                         else " (fits L2): L2 flushed before every step, per-step events")}
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x2" if tc else prec_name.replace("fp", "f"), "data": "synthetic",
        "config": cfg, "roofline": roof,
        "comparator": {"kernel": "plain FP64 quadrature nest", "value": naive_rate, "unit": METRIC,
                       "elements": En, "ms_per_step": ms_naive, "speedup": value / world / naive_rate},
        "e2e": {"value": E * world / (e2e_ms * 1e-3), "unit": METRIC,
                "h2d_bytes_per_step": E * (96 + 8 * fea.coeff_len(form, p)), "d2h_bytes_per_step": E * n * n * esz,
                "ms_per_step": e2e_ms},
        "gpu_launches": args.steps, "clocks": clk.summary(), "gflops": flops / (ms * 1e-3) / 1e9,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(form, p, coords, coeffs)
    return line


VECTOR_WORKLOADS = {
    # name: (form, degree, elements) -- element vectors of the linear forms
    "helmholtz_load_p2_1M": (1, 2, 1_000_000),
    "neohookean_residual_p2_500k": (3, 2, 500_000),
}


def run_vector(args, fea, torch, barrier, max_over_ranks, world, rank, local):
    """Element vectors (fea_assemble_vector): the Helmholtz load vector or the
    Neo-Hookean residual of the matrix workloads' inputs."""
    from paper_1604_05872_gb300 import inputs
    form, p, E0 = VECTOR_WORKLOADS[args.workload]
    E = args.elements or E0
    coords, coeffs = inputs.workload(form, p, E, seed=inputs.SEED + rank)
    c = torch.from_numpy(coords).cuda()
    fc = torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    f32 = bool(args.out_f32)
    n = fea.local_dim(form, p)
    out = torch.empty((E, n), dtype=torch.float32 if f32 else torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        fea.assemble_vector(form, p, c, fc, out=out, out_f32=f32)
    fea.sync()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            fea.assemble_vector(form, p, c, fc, out=out, out_f32=f32)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    fea.sync()
    ms_max = max_over_ranks(ms)
    ns = (p + 1) * (p + 2) * (p + 3) // 6
    Q = fea.quad_points(form if form == 3 else 0, p)
    esz = 4 if f32 else 8
    bytes_elem = 96 + 8 * fea.coeff_len(form, p) + esz * n
    # executed FP32 flops and FP64 lane-instructions per element (estimates of the kernels' loop nests)
    if form == 1:
        flops, f64 = 2 * ns * ns + ns, 20
    else:
        flops, f64 = Q * (2 * 9 * ns + 2 * 27 + 2 * 27 + 2 * 27 + 18 * ns), 30 + NEO_POINT_FP64 * Q
    hbm, peak_kind = peaks()
    alg_bytes, fl, f64t = E * bytes_elem, E * flops, E * f64
    t_hbm, t_f32, t_f64 = alg_bytes / (hbm * 1e9), fl / (FP32_PEAK_TFLOPS * 1e12), f64t / (FP64_PEAK_TINSTR * 1e12)
    if t_hbm >= max(t_f32, t_f64):
        roof = {"bound": "hbm", "achieved": alg_bytes / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_kind": peak_kind}
    elif t_f64 >= t_f32:
        roof = {"bound": "alu", "achieved": f64t / (ms * 1e-3) / 1e12, "peak": FP64_PEAK_TINSTR,
                "unit": "T FP64 lane-instructions/s", "peak_kind": "derived: FP64 lanes x clock"}
    else:
        roof = {"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "peak_kind": "derived: FP32 lanes x clock"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    full = E == VECTOR_WORKLOADS[args.workload][2]
    roof["traffic"] = profiled_traffic(args.workload) if full and not f32 else None
    roof["alg_bytes_per_launch"] = alg_bytes
    roof["bound_times_ms"] = {"hbm": t_hbm * 1e3, "fp32": t_f32 * 1e3, "fp64": t_f64 * 1e3}
    line = {
        "metric": "element vectors/s", "value": E * world / (ms_max * 1e-3), "unit": "element vectors/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "form": ["mass", "helmholtz", "elasticity", "neohookean"][form],
                   "degree": p, "elements": E, "quad_points": Q, "local_vector": "%d %s" % (n, "f32" if f32 else "f64"),
                   "l2": "inputs+outputs %.0f MB per step%s" % (alg_bytes / 1e6, " > 129 MB L2; no flush"
                                                             if alg_bytes > 129e6 else " (fits L2)")},
        "roofline": roof, "gpu_launches": args.steps, "clocks": clk.summary(), "e2e": None,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        nsamp = min(E, 1_000_000 if form == 1 else 50_000)
        t0 = time.perf_counter()
        if form == 1:
            oracle.load_vector(p, coords[:nsamp], coeffs[:nsamp])
        else:
            oracle.neohookean_residual(p, coords[:nsamp], coeffs[:nsamp])
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": nsamp / dt, "unit": "element vectors/s", "cores": 1, "kind": "oracle",
                                "sample": "first %d elements, FP64 loop nest, one core, %.2f s" % (nsamp, dt)}
    return line


def bernstein_flops(p):
    """Executed FP32 flops per element of the sum-factorised Bernstein kernel: the
    six 1-D passes (f at the points, then the moments of degree 2p), the mass
    entries (one product each) and the six-term pre-evaluated stiffness, 2 flops
    per multiply-add."""
    m = (3 * p + 2) // 2
    n2 = 2 * p
    ns = (p + 1) * (p + 2) * (p + 3) // 6
    pairs1 = [(a3, a2) for a3 in range(p + 1) for a2 in range(p - a3 + 1)]
    e1 = sum(p - a3 - a2 + 1 for a3, a2 in pairs1) * m
    e2 = sum(p - a3 + 1 for a3 in range(p + 1)) * m * m
    e3 = m ** 3 * (p + 1) + m ** 3
    m1 = (n2 + 1) * m * m * m
    m2 = (n2 + 1) * (n2 + 2) // 2 * m * m
    m3 = (n2 + 1) * (n2 + 2) * (n2 + 3) // 6 * m
    return 2 * (e1 + e2 + e3 + m1 + m2 + m3) + ns * ns * (1 + 2 * 6)


def run_bernstein(args, fea, torch, barrier, max_over_ranks, world, rank, local):
    """Helmholtz P4 in the Bernstein-Bezier basis by sum factorisation
    (fea_assemble_bernstein), 200 000 elements; the Lagrange pre-evaluated
    kernel on the same elements is timed beside it for comparison."""
    from paper_1604_05872_gb300 import inputs
    p, E = 4, args.elements or 200_000
    coords, _ = inputs.workload(1, p, E, seed=inputs.SEED + rank)
    ns = (p + 1) * (p + 2) * (p + 3) // 6
    cb = np.random.Generator(np.random.PCG64(inputs.SEED + 11 + rank)).uniform(-1.0, 1.0, (E, ns))
    c, fb = torch.from_numpy(coords).cuda(), torch.from_numpy(cb).cuda()
    f32 = bool(args.out_f32)
    out = torch.empty((E, ns, ns), dtype=torch.float32 if f32 else torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        fea.sync()
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            fn()
        ev1.record(stream)
        barrier()
        fea.sync()
        return ev0.elapsed_time(ev1) / steps

    with ClockSampler(local) as clk:
        ms = timed(lambda: fea.assemble_bernstein(1, p, c, fb, out=out, out_f32=f32), args.steps)
    ms_lagrange = timed(lambda: fea.assemble(1, p, c, fb, out=out, out_f32=f32), max(3, args.steps // 4))
    ms_max = max_over_ranks(ms)
    esz = 4 if f32 else 8
    alg_bytes = E * (96 + 8 * ns + esz * ns * ns)
    flops = E * bernstein_flops(p)
    hbm, peak_kind = peaks()
    t_hbm, t_f32 = alg_bytes / (hbm * 1e9), flops / (FP32_PEAK_TFLOPS * 1e12)
    if t_hbm >= t_f32:
        roof = {"bound": "hbm", "achieved": alg_bytes / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_kind": peak_kind}
    else:
        roof = {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "peak_kind": "derived: FP32 lanes x clock"}
    roof.update({"frac": roof["achieved"] / roof["peak"], "traffic": None, "alg_bytes_per_launch": alg_bytes,
                 "bound_times_ms": {"hbm": t_hbm * 1e3, "fp32": t_f32 * 1e3}})
    pl = fea.plan(1, p)
    return {
        "metric": METRIC, "value": E * world / (ms_max * 1e-3), "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "form": "helmholtz", "degree": p, "elements": E,
                   "basis": "Bernstein-Bezier", "method": "sum factorisation of the moments of f over the collapsed rule",
                   "local_matrix": "%dx%d %s" % (ns, ns, "f32" if f32 else "f64"),
                   "flops_per_element": bernstein_flops(p), "lagrange_pre_flops_per_element": pl["flops_run"],
                   "l2": "inputs+outputs %.0f MB per step > 129 MB L2; no flush" % (alg_bytes / 1e6)},
        "comparator": {"kernel": "Lagrange basis, pre-evaluated (fea_assemble, same elements)",
                       "ms_per_step": ms_lagrange, "value": E / (ms_lagrange * 1e-3), "unit": METRIC},
        "roofline": roof, "gpu_launches": args.steps, "clocks": clk.summary(), "e2e": None,
    }


def run_global(args, fea, torch, barrier, max_over_ranks, world, rank, local):
    """Local and global assembly together (the paper times them jointly): Helmholtz P2 on a
    conforming mesh of the unit cube (55^3 cubes x 6 tetrahedra = 998 250 elements, 1.37 M DOFs;
    --elements picks the nearest cube mesh for profiling).
    One step: zero the CSR values, then fea_assemble_csr_combined (element matrices summed per
    distinct CSR position of a tile in shared memory, one FP64 atomic per position, never
    stored; the positions and their grouping computed once per mesh).  Also timed: the one-pass
    kernel with one atomic per entry (fea_assemble_csr), the two-pass form (fea_assemble, then
    fea_scatter_add_csr_mapped), the scatters alone and symmetric storage."""
    from paper_1604_05872_gb300 import inputs
    m = 55 if not args.elements else max(2, int(round((args.elements / 6) ** (1 / 3))))  # cubes per edge
    coords, dofs, nd = inputs.box_mesh(m, 2, jitter=0.1, seed=inputs.SEED + rank)
    E = coords.shape[0]
    rng = np.random.Generator(np.random.PCG64(inputs.SEED + 7 + rank))
    f = inputs.random_coeffs(1, 2, E, rng)
    t0 = time.perf_counter()
    row_ptr, col_idx = fea.csr_pattern(dofs, nd)
    t_pattern = time.perf_counter() - t0
    c, fc = torch.from_numpy(coords).cuda(), torch.from_numpy(inputs.coeff_array(1, 2, f)).cuda()
    dd, rp, ci = (torch.from_numpy(x).cuda() for x in (dofs, row_ptr, col_idx))
    elem = fea.empty_out(1, 2, E)
    nnz = col_idx.shape[0]
    vals = torch.zeros(nnz, dtype=torch.float64, device="cuda")
    smap = fea.csr_scatter_map(dd, rp, ci)  # CSR positions, once per mesh
    t0 = time.perf_counter()
    host_plan = fea.csr_combine_plan(smap, nnz)  # grouping per tile, once per mesh
    t_plan = time.perf_counter() - t0
    plan = torch.from_numpy(host_plan).cuda()
    tile = int(host_plan[2])
    ntiles = (E + tile - 1) // tile
    toff = host_plan[4:4 + 2 * (ntiles + 1)].view(np.int64)
    positions = int(host_plan[toff[:-1]].astype(np.int64).sum())  # one FP64 atomic each
    stream = torch.cuda.current_stream()

    def step():
        vals.zero_()
        fea.assemble_csr_combined(1, 2, c, fc, plan, vals)

    def one_pass_map():
        vals.zero_()
        fea.assemble_csr(1, 2, c, fc, smap, vals)

    def two_pass():
        fea.assemble(1, 2, c, fc, out=elem)
        vals.zero_()
        fea.scatter_add_csr_mapped(smap, elem, vals)

    def timed(fn, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / steps

    for _ in range(args.warmup):
        step()
        one_pass_map()
        two_pass()
    fea.sync()
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for _ in range(args.steps):
            step()
        ev[1].record(stream)
        barrier()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    # the combined kernel alone (it accumulates: the same work every launch), the one-pass step
    # with one atomic per entry and its kernel, the two-pass step, and its scatter with
    # precomputed positions and with the per-entry search
    ms_kernel = timed(lambda: fea.assemble_csr_combined(1, 2, c, fc, plan, vals), args.steps)
    ms_map_kernel = timed(lambda: fea.assemble_csr(1, 2, c, fc, smap, vals), args.steps)
    ms_map = timed(one_pass_map, args.steps)
    ms_two = timed(two_pass, args.steps)
    # symmetric storage: the upper triangle only (55 of the 100 entries of each element matrix)
    ur, uc = fea.csr_pattern(dofs, nd, upper=True)
    umap = fea.csr_scatter_map(dd, torch.from_numpy(ur).cuda(), torch.from_numpy(uc).cuda(), upper=True)
    uplan = torch.from_numpy(fea.csr_combine_plan(umap, uc.shape[0])).cuda()
    uvals = torch.zeros(uc.shape[0], dtype=torch.float64, device="cuda")

    def sym_step():
        uvals.zero_()
        fea.assemble_csr_combined(1, 2, c, fc, uplan, uvals)

    def sym_map_step():
        uvals.zero_()
        fea.assemble_csr(1, 2, c, fc, umap, uvals)

    for _ in range(args.warmup):
        sym_step()
        sym_map_step()
    ms_sym = timed(sym_step, args.steps)
    ms_sym_map = timed(sym_map_step, args.steps)
    ms_scatter = timed(lambda: fea.scatter_add_csr_mapped(smap, elem, vals), args.steps)
    ms_search = timed(lambda: fea.scatter_add_csr(dd, elem, rp, ci, vals), max(1, args.steps // 4))
    fea.sync()
    ms_max = max_over_ranks(ms)
    # algorithmic bytes of the combined kernel: coordinates and coefficients (176 B/element), the
    # plan (positions, tile-entry indices, headers), one read and one write of every CSR value;
    # the step adds the zeroing of the values (8 B per entry)
    plan_bytes = 4 * host_plan.shape[0]
    kernel_bytes = E * 176 + plan_bytes + nnz * 16
    step_bytes = kernel_bytes + nnz * 8
    map_kernel_bytes = E * (176 + 100 * smap.element_size()) + nnz * 16
    hbm, peak_kind = peaks()
    roof = {"bound": "hbm", "kernel": "pre_combine_kernel<1, 2>",
            "achieved": kernel_bytes / (ms_kernel * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
            "peak_kind": peak_kind, "traffic": profiled_traffic(args.workload),
            "alg_bytes_per_launch": kernel_bytes, "kernel_ms": ms_kernel,
            "fp64_atomics_per_launch": positions, "fp64_atomics_per_s": positions / (ms_kernel * 1e-3),
            "step_achieved": step_bytes / (ms * 1e-3) / 1e9, "step_alg_bytes": step_bytes,
            "map_kernel_ms": ms_map_kernel,
            "map_kernel_frac": map_kernel_bytes / (ms_map_kernel * 1e-3) / 1e9 / hbm}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["step_frac"] = roof["step_achieved"] / roof["peak"]
    line = {
        "metric": METRIC, "value": E * world / (ms_max * 1e-3), "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "form": "helmholtz", "degree": 2, "elements": E, "dofs": nd,
                   "nnz": nnz, "local_matrix": "10x10, never stored",
                   "global": "CSR f64; a tile's entries summed per distinct position in shared memory, one "
                             "FP64 atomic per position (%d tiles of %d elements, %.1f atomics per element)"
                             % (ntiles, tile, positions / E),
                   "plan_bytes": plan_bytes, "plan_host_s": t_plan, "pattern_host_s": t_pattern,
                   "one_pass_map_ms": ms_map, "two_pass_ms": ms_two, "scatter_ms": ms_scatter,
                   "scatter_with_search_ms": ms_search,
                   "symmetric_storage_ms": ms_sym, "symmetric_storage_map_ms": ms_sym_map,
                   "symmetric_nnz": int(uc.shape[0]),
                   "l2": "%.0f MB per step > 129 MB L2; no flush" % (step_bytes / 1e6)},
        "roofline": roof, "gpu_launches": args.steps, "clocks": clk.summary(), "e2e": None,
    }
    return line


def run_stream(args, fea, torch, barrier, max_over_ranks, world, local):
    """64 uneven requests (4 forms x P1-P4, 2M elements) in one persistent,
    graph-captured launch; flop-count choices, then (with --tuning) the MLP's."""
    from paper_1604_05872_gb300 import inputs
    reqs = inputs.stream_requests()
    built, total, alg_bytes, t_bound = [], 0, 0, 0.0
    hbm, peak_kind = peaks()
    for k, (form, p, E) in enumerate(reqs):
        coords, coeffs = inputs.workload(form, p, E, seed=inputs.SEED + 100 + k, anisotropic=(form == 2))
        c = torch.from_numpy(coords).cuda()
        f = None if form == 0 else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
        built.append((form, p, c, f, fea.empty_out(form, p, E)))
        total += E

    bf16, _ = bf16_peak()
    prec_name = "bf16x2" if args.precision in ("auto", "bf16x2") else "fp32"
    prec = fea.PREC_BF16X2 if prec_name == "bf16x2" else fea.PREC_FP32

    def bound_time():
        tb, byt = 0.0, 0
        for form, p, c, f, o in built:
            pl = fea.plan(form, p, precision=prec)
            tc = pl["threads"] != 256
            E = c.shape[0]
            b = E * pl["bytes"]
            byt += b
            if tc:
                tb += max(b / (hbm * 1e9), E * tc_flops_per_element(form, p) / (bf16 * 1e12),
                          E * (30 + NEO_POINT_FP64_TC * pl["quad_points"]) / (FP64_PEAK_TINSTR * 1e12))
            else:
                tb += max(b / (hbm * 1e9), E * pl["flops_run"] / (FP32_PEAK_TFLOPS * 1e12),
                          E * fp64_ops_per_element(form, p, pl["variant"], pl["quad_points"]) / (FP64_PEAK_TINSTR * 1e12))
        return tb, byt

    def timed(steps, fused=False):
        for _ in range(args.warmup):
            fea.assemble_batch(built, fused=fused, precision=fea.PREC_FP32 if fused else prec)
        fea.sync()
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            fea.assemble_batch(built, fused=fused, precision=fea.PREC_FP32 if fused else prec)
        ev1.record()
        barrier()
        fea.sync()
        return ev0.elapsed_time(ev1) / steps

    fea.tune_clear()
    t_bound, alg_bytes = bound_time()
    with ClockSampler(local) as clk:
        ms_flop = timed(args.steps)
    ms_fused = timed(args.steps, fused=True)
    result = {"flop_choice_ms": ms_flop, "fused_kernel_ms": ms_fused}
    ms = ms_flop
    choice = "flop-count (Algorithm 3, default tiles)"
    if args.tuning and os.path.exists(args.tuning):
        from paper_1604_05872_gb300 import tuning
        _, model = tuning.load(args.tuning)
        for form in range(4):
            for p in range(1, 5):
                tuning.choose(model, form, p)
        ms_mlp = timed(args.steps)
        t_bound_mlp, _ = bound_time()
        result.update({"mlp_choice_ms": ms_mlp, "mlp_gain": ms_flop / ms_mlp})
        if ms_mlp < ms_flop:
            ms, choice, t_bound = ms_mlp, "learned MLP cost model", t_bound_mlp
        fea.tune_clear()
    ms_max = max_over_ranks(ms)
    return {
        "metric": METRIC, "value": total * world / (ms_max * 1e-3), "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "stream_64req_2M", "requests": len(reqs), "elements": total, "choice": choice,
                   "contraction": prec_name + (" (split-BF16 tensor cores for the Neo-Hookean P2 requests, FP32 elsewhere)"
                                               if prec_name == "bf16x2" else ""),
                   "launch": "one replayed CUDA graph per step: each request's persistent kernel, 4 concurrent branches"},
        "roofline": {"bound": "mixed", "achieved": t_bound * 1e3, "peak": ms, "unit": "ms (sum of per-request bound times / measured)",
                     "frac": t_bound * 1e3 / ms, "traffic": None, "alg_bytes_per_launch": alg_bytes,
                     "peak_kind": peak_kind},
        "stream": result, "gpu_launches": args.steps, "clocks": clk.summary(), "e2e": None,
    }


if __name__ == "__main__":
    main()
