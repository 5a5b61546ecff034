#!/usr/bin/env python
"""Throughput of the MPO Lindblad Trotter step on GB300.

Workload (default ``chain20_chi256``): N=20 open chain with the seeded
couplings of the precision-comparison model (J_b~U[0.05,0.15],
Omega~U[0.3,0.7], g0_i~U[0.005,0.02], g2_i~U[0.01,0.03], h_z alternating 0,1),
chi_max = 256 saturated from the first step (seeded random MPO start), cutoff
1e-10, dt = 0.02, second-order Trotter: 29 two-site gate applications per step,
most of them on bond matrices of up to 1024 x 1024.

A step = one mpdo_trotter_step(1) over the whole batch (merge, gate, weight,
QR + Jacobi SVD, truncation, reconstruction for every op, trace forcing).
``value`` = gate applications per second of the batched mixed-precision path
(device-timed, inputs resident); ``fp64_path`` = the same steps on the FP64
path, ``fp64_per_gate`` = the FP64 path with one op in flight at a time (the
plain per-gate path), ``speedup_mixed_vs_fp64`` = their ratio to ``value``;
``batched`` = the 64-instance N=16 workload; ``e2e`` = the headline metric
through the C ABI with the state uploaded from host memory and observables
read back each step.

--gpus N > 1 runs N independent replicas (one per rank, launched by torchrun):
the method has no exchange step between instances.
``--impl reference`` times the CPU oracle on the machine's host cores: each step is
one gate application of the workload (ops taken in step order, cycling), with
the oracle's LAPACK SVD route (numpy, all host cores), the paper's own
threaded-LAPACK design.  ``cpu_baseline`` (in the GPU line) times the same
route on 5 ops after one warm-up op, and ``cpu_baseline_plain`` one op of the
oracle's plain C Jacobi on one thread.
``--probe-peaks`` measures the FP64 / FP32 / TF32 GEMM rates with cuBLAS.
``adjoint`` (``--adjoint-steps``, default 1): one gradient of the observables
on the N=24 ring at chi = 256 (checkpointed forward, then recompute and
backward), timed next to plain steps from the same state.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_PEAK_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (recipe table, nominal)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="chain20_chi256")
    ap.add_argument("--precision", default="both", choices=["fp64", "mixed", "both"])
    ap.add_argument("--mixed-kind", default="tf32", choices=["tf32", "bf16"],
                    help="tensor kind of the mixed path's slice products (MPDO_MIXED_TF32 / MPDO_MIXED_BF16X3)")
    ap.add_argument("--per-gate-steps", type=int, default=1,
                    help="timed steps of the FP64 path with one op in flight (0: skip)")
    ap.add_argument("--batched-steps", type=int, default=1,
                    help="timed steps of the 64-instance batched workload (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-ops", type=int, default=5, help="timed oracle ops of every op shape in cpu_baseline")
    ap.add_argument("--no-cpu-plain", action="store_true", help="skip the plain C Jacobi op")
    ap.add_argument("--oracle-svd", default="lapack", choices=["lapack", "jacobi"],
                    help="SVD route of --impl reference")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--probe-peaks", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default Jacobi block rule")
    ap.add_argument("--no-graph", action="store_true", help="skip the graph-replayed steps")
    ap.add_argument("--no-observables", action="store_true",
                    help="skip the observables timing on the 4x10 snake at chi 512")
    ap.add_argument("--precond-rho", type=float, default=0.0,
                    help="mixed path: largest FP32 rotation at which the preconditioning sweeps stop (0: default)")
    ap.add_argument("--qr-blocked", action="store_true",
                    help="mixed path: blocked Householder QR (tensor-core trailing updates) instead of the column QR")
    ap.add_argument("--adjoint-steps", type=int, default=1,
                    help="Trotter steps of the timed gradient on the N=24 ring at chi=256 (0: skip)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# Schmidt-value grading of the synthetic start: exp(-DECAY * r) on bond index r,
# i.e. about 6e-3 between the first and the 256th value, so that the 1e-10
# cutoff never binds before chi_max = 256 and every inner bond of the chain
# stays saturated through the timed steps
DECAY = 0.02


def make_workload(name):
    """(workload, [(dims, tensors)] per instance, chi_cap)."""
    import workloads as W
    if name == "batch64_chain16":
        # 64 independent N=16 chains, chi_max drawn from {32, 64, 128, 256} per
        # instance, each started at its own saturated chi (seeded random MPO)
        wl = W.batch64_chain16()
        states = [W.random_mpo_state(wl.n, int(wl.chi_max[b]), seed=2203058712 + 100 + b, decay=DECAY)
                  for b in range(wl.batch)]
        return wl, states, 256
    if name == "snake4x10_chi512":
        # the 4x10 grid on a snake path at its chi_max = 512 (bond ranges 1, 3,
        # 5, 7 through swap chains), started at saturated chi
        wl = W.grid4x10_snake()
        return wl, [W.random_mpo_state(wl.n, 512, seed=2203058712 + 3, decay=DECAY)], 512
    table = {"chain20_chi256": (256, DECAY), "chain20_chi256_flat": (256, 0.0),
             "chain20_chi128": (128, DECAY), "chain20_chi64": (64, DECAY),
             "chain10_chi256": (256, DECAY)}
    if name not in table:
        raise SystemExit(f"unknown workload {name}")
    chi, decay = table[name]
    wl = W.chain20_precision(chi_max=chi)
    if name.startswith("chain10"):   # small case of the same model (profiling)
        wl = W.uniform_model("chain10_chi256", 10, W.chain_bonds(10), chi_max=chi, cutoff=1e-10, dt=0.02)
    return wl, [W.random_mpo_state(wl.n, chi, seed=2203058712 + 1, decay=decay)], chi


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        import statistics
        sm, mx, reasons = [], [], set()
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def cpu_info():
    """Host CPU model and core count (recorded next to every CPU number)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"nproc": os.cpu_count(), "model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def oracle_ops(wl, dims, tens, count, warm, svd_impl, full_size_only=False):
    """Time the oracle's two-site update on the workload's ops in step order
    (cycling), each from the saturated start state; full_size_only keeps the
    ops whose bond matrix is (4 chi_max) x (4 chi_max).  Returns (per-op seconds
    of the timed ops, description)."""
    import numpy as np
    from oracle import schedule, tebd
    layers = schedule.step_layers(wl.n, wl.bonds)
    gates = tebd.build_gates(wl, 0, layers, wl.dt)
    ops = [(op[1], G) for L, gl in zip(layers, gates) for op, G in zip(L, gl)]
    st = tebd.MPOState(tens, [np.ones(d) for d in dims[1:-1]])
    cap = int(wl.chi_max[0])
    if full_size_only:
        ops = [(p, G) for (p, G) in ops if dims[p] == cap and dims[p + 2] == cap] or ops
    times, sizes = [], []
    for r in range(warm + count):
        p, G = ops[r % len(ops)]
        s = st.copy()
        t0 = time.perf_counter()
        s.apply(p, G, cap, float(wl.cutoff[0]), svd_impl=svd_impl)
        dt = time.perf_counter() - t0
        if r >= warm:
            times.append(dt)
            sizes.append(f"{4 * dims[p]}x{4 * dims[p + 2]}")
    route = ("oracle MPO-TEBD update, LAPACK gesdd SVD through numpy (threaded BLAS)" if svd_impl == "lapack"
             else "oracle MPO-TEBD update, plain C one-sided Jacobi SVD, one thread")
    return times, f"{len(times)} ops of the step in order after {warm} warm-up (bond matrices {', '.join(sizes)}); {route}"


def oracle_step_estimate(wl, dims, tens, reps, warm, svd_impl):
    """A Trotter step of the oracle, estimated from a bounded sample: the step's
    ops grouped by bond-matrix shape, one op of every shape timed per rep (after
    `warm` untimed ops of the largest shape), each shape's mean time weighted by
    its count in the step.  Returns (ops per step, estimated seconds per step,
    description)."""
    import numpy as np
    from oracle import schedule, tebd
    layers = schedule.step_layers(wl.n, wl.bonds)
    gates = tebd.build_gates(wl, 0, layers, wl.dt)
    ops = [(op[1], G) for L, gl in zip(layers, gates) for op, G in zip(L, gl)]
    st = tebd.MPOState(tens, [np.ones(d) for d in dims[1:-1]])
    cap = int(wl.chi_max[0])
    classes = {}
    for p, G in ops:
        classes.setdefault((4 * dims[p], 4 * dims[p + 2]), []).append((p, G))

    def run(p, G):
        s = st.copy()
        t0 = time.perf_counter()
        s.apply(p, G, cap, float(wl.cutoff[0]), svd_impl=svd_impl)
        return time.perf_counter() - t0
    big = max(classes, key=lambda k: k[0] * k[1])
    for _ in range(warm):
        run(*classes[big][0])
    mean = {k: sum(run(*v[0]) for _ in range(max(1, reps))) / max(1, reps) for k, v in classes.items()}
    est = sum(mean[k] * len(v) for k, v in classes.items())
    route = ("oracle MPO-TEBD update, LAPACK gesdd SVD through numpy (threaded BLAS)" if svd_impl == "lapack"
             else "oracle MPO-TEBD update, plain C one-sided Jacobi SVD, one thread")
    mix = ", ".join(f"{len(v)} x {k[0]}x{k[1]}" for k, v in sorted(classes.items(), key=lambda kv: -len(kv[1])))
    what = (f"one step of {len(ops)} ops estimated from {max(1, reps)} timed op(s) of each bond-matrix shape "
            f"after {warm} warm-up op(s), weighted by the step's mix ({mix}); {route}")
    return len(ops), est, what


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl, states, cap = make_workload(args.workload)
    b = next(i for i in range(wl.batch) if int(wl.chi_max[i]) == cap)   # an instance at full chi
    dims, tens = states[b]
    threads = os.cpu_count() if args.oracle_svd == "lapack" else 1
    if args.oracle_svd == "lapack":
        # the whole step's op mix (a plain C Jacobi op of full size takes about a minute: that
        # route times full-size ops only)
        n_ops, est, what = oracle_step_estimate(wl.instance(b), dims, tens, args.steps, args.warmup, "lapack")
        v, ms_step = n_ops / est, 1e3 * est
    else:
        times, what = oracle_ops(wl.instance(b), dims, tens, args.steps, args.warmup, args.oracle_svd,
                                 full_size_only=True)
        v, ms_step = len(times) / sum(times), 1e3 * sum(times) / len(times)
    info = cpu_info()
    line = {"impl": "reference", "metric": "gate_applications_per_sec", "value": v,
            "unit": "gate-applications/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "oracle": what,
                       "step": ("one Trotter step (estimated)" if args.oracle_svd == "lapack"
                                else "one full-size gate application")},
            "cpu_baseline": {"value": v, "unit": "gate-applications/s", "cores": threads, "kind": "oracle",
                             "sample": what, "cpu": info},
            "e2e": {"value": v, "unit": "gate-applications/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def cpu_baseline_subprocess(args, svd_impl, count, warm):
    """The oracle sample in a child process: LAPACK route on every host core,
    or the plain C Jacobi route with one BLAS thread."""
    env = dict(os.environ)
    if svd_impl == "jacobi":
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = "1"
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", str(count), "--warmup",
           str(warm), "--workload", args.workload, "--oracle-svd", svd_impl]
    try:
        out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900).stdout
        line = json.loads(out.strip().splitlines()[-1])
        return line["cpu_baseline"]
    except Exception as ex:  # baseline failure must not hide the GPU number
        return {"value": None, "unit": "gate-applications/s", "cores": None, "kind": "oracle",
                "sample": f"failed: {ex}"}


# ---------------------------------------------------------------------------
def probe_peaks():
    import torch
    res = {}

    def best(fn, it=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        b = 1e9
        for _ in range(it):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            b = min(b, s.elapsed_time(e) / 1e3)
        return b
    torch.backends.cuda.matmul.allow_tf32 = False
    for dt, n, key in [(torch.float64, 8192, "fp64_dgemm_tflops"), (torch.float32, 8192, "fp32_sgemm_tflops")]:
        a = torch.randn(n, n, device="cuda", dtype=dt)
        b = torch.randn(n, n, device="cuda", dtype=dt)
        res[key] = 2 * n ** 3 / best(lambda: a @ b) / 1e12
    torch.backends.cuda.matmul.allow_tf32 = True
    a = torch.randn(8192, 8192, device="cuda")
    b = torch.randn(8192, 8192, device="cuda")
    res["tf32_gemm_tflops"] = 2 * 8192 ** 3 / best(lambda: a @ b) / 1e12
    res["how"] = "torch.matmul 8192^3, best of 10, CUDA events"
    print(json.dumps(res))


# ---------------------------------------------------------------------------
def run_arm(args, precision, world, dist, local, workload=None, steps=None, warmup=None, max_slots=0,
            graph=True, e2e_steps=None, autotune=True):
    """Time Trotter steps of one precision on one workload; returns a result dict."""
    import numpy as np
    import torch
    from paper_2203_05871_gb300 import FP64, MIXED_BF16X3, MIXED_TF32, Solver

    workload = workload or args.workload
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    e2e_steps = args.e2e_steps if e2e_steps is None else e2e_steps
    wl, states, cap = make_workload(workload)
    stream = torch.cuda.Stream()
    mixed = MIXED_BF16X3 if args.mixed_kind == "bf16" else MIXED_TF32
    s = Solver(wl.n, batch=wl.batch, chi_cap=cap, stream=stream,
               precision=FP64 if precision == "fp64" else mixed, max_slots=max_slots,
               qr_blocked=args.qr_blocked, precond_rho=args.precond_rho)
    s.build_gates(wl)
    tuned = None
    if autotune and not args.no_autotune:
        from paper_2203_05871_gb300.mpdo import saturated_classes
        cls = saturated_classes(wl.n, cap)
        tuned = {f"{a}x{b}": [int(x) for x in blk] for (a, b), blk in zip(cls, s.autotune(cls))}
    for b, (dims, tens) in enumerate(states):
        s.set_state(b, dims, tens)
    n_ops, n_swaps, _ = s.op_counts()
    n_ops_all = n_ops * wl.batch
    for _ in range(warmup):
        s.step(1)
    torch.cuda.synchronize()
    chi_warm = s.status()["chi"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    s.profile(True)
    s.profile_read(reset=True)
    ms = 0.0
    with ClockSampler(local) as clk:
        for _ in range(steps):
            flush.fill_(1.0)                       # L2 flush between timed steps
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(1)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
    prof = s.profile_read(reset=True)
    s.profile(False)
    graph_ms = None
    if graph:
        # the same steps replayed as a captured CUDA graph (first call captures)
        s.step(1, graph=True)
        graph_ms = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(1, graph=True)
            e1.record(stream)
            torch.cuda.synchronize()
            graph_ms += e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    st = s.status()
    # end to end through the C ABI from host buffers (state in, observables out)
    flat_bytes = sum(int(np.asarray(t).size) for (_, tens) in states for t in tens) * 8
    e2e_ms = 0.0
    for _ in range(e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b, (dims, tens) in enumerate(states):
            s.set_state(b, dims, tens)
        s.step(1)
        s.measure_1q(range(wl.n), "Z")
        e2e_ms += (time.perf_counter() - t0) * 1e3
    s.close()
    return {"wl": wl, "cap": cap, "n_ops": n_ops_all, "n_swaps": n_swaps, "ms": ms, "steps": steps,
            "graph_ms": graph_ms, "prof": prof, "status": st, "tuned": tuned, "chi_warm": chi_warm,
            "clocks": clk.summary(), "e2e_ms": e2e_ms, "e2e_steps": e2e_steps, "flat_bytes": flat_bytes}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


SLICE_PRODUCTS = 21   # slice pairs (t, u), t + u <= 5, per useful multiply-add of the tensor-core products


def contraction_roofline(prof, kind):
    """The tensor-core contractions (merge + reconstruct, oz_gemm_kernel with its
    slicing kernels) against the tensor peak of their kind: executed flops = 21
    slice products per useful flop (the hardware's work), with the useful rate
    beside it."""
    fl = prof["merge_gate"]["flops"] + prof["reconstruct"]["flops"]
    ms = prof["merge_gate"]["ms"] + prof["reconstruct"]["ms"]
    bf16 = measured_peaks().get("bf16_tflops")
    base = bf16 if bf16 else 1900.0
    peak = base if kind == "bf16" else base * 1.1 / 2.25
    useful = fl / (ms / 1e3) / 1e12 if ms > 0 else None
    achieved = useful * SLICE_PRODUCTS if useful else None
    return {"kernel": "oz_gemm_kernel (merge + reconstruct, incl. slicing and the gate/weight kernel)",
            "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None, "traffic": None, "useful_tflops": useful,
            "note": "achieved = 21 slice products x useful flops (32 cl cm cr + 512 cl cr merge, 32 cl cr k "
                    "reconstruct) / CUDA-event time of the merge and reconstruct stages; peak = measured bf16 burst"
                    + (" x 1.1/2.25 (nominal TF32/BF16)" if kind != "bf16" else "") + ("" if bf16 else ", of fallback")}


def qr_roofline(prof):
    """Householder QR with column pivoting against the nominal FP64 peak."""
    q = prof["qr"]
    achieved = q["flops"] / (q["ms"] / 1e3) / 1e12 if q["ms"] > 0 else None
    return {"kernel": "qr_kernel (Householder, column pivoting)", "bound": "alu", "achieved": achieved,
            "peak": FP64_PEAK_NOMINAL_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_NOMINAL_TFLOPS if achieved else None, "traffic": None,
            "note": "flops 4 m n r - 2 (m + n) r^2 + 4/3 r^3 per op (r = min(m, n)); peak = nominal FP64"}


def run_observables(args, local, reps=5):
    """Measurement (a12) and the global quantities on the 4x10 snake at
    chi_max = 512 (N = 40, bonds saturated from position 4 inward, seeded
    random MPO): every <Z_i>, every connected <Z_i Z_j> (780 pairs), S2 and the
    central OSEE, each timed with CUDA events on the solver's stream after
    warm-up.  The sites (336 MB) exceed L2, so no flush is needed."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2203_05871_gb300 import FP64, Solver

    wl = W.grid4x10_snake()
    n, chi = wl.n, 512
    dims, tens = W.random_mpo_state(n, chi, seed=2203058712 + 3, decay=DECAY)
    stream = torch.cuda.Stream()
    s = Solver(n, batch=1, chi_cap=chi, stream=stream, precision=FP64, max_slots=2)
    s.build_gates(wl)
    s.set_state(0, dims, tens)
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    o1 = torch.empty((1, n), dtype=torch.float64, device="cuda")
    o2 = torch.empty((1, len(pairs)), dtype=torch.float64, device="cuda")
    calls = {"z_all": lambda: s.measure_1q(range(n), "Z", out=o1),
             "zz_connected_all_pairs": lambda: s.measure_2q(pairs, "ZZ", connected=True, out=o2),
             "renyi2": lambda: s.renyi2(),
             "osee_central": lambda: s.osee()}
    res = {}
    with ClockSampler(local) as clk:
        for name, fn in calls.items():
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            res[name] = {"ms": a.elapsed_time(b) / reps}
    d = np.asarray(dims, dtype=np.float64)
    slice_bytes = float(np.sum(d[:-1] * d[1:])) * 8.0        # one Pauli slice of every site
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    # <Z_i> for all i: left and right I-environments and one Z slice per site
    b1 = 3.0 * slice_bytes
    res["z_all"]["roofline"] = {"bound": "hbm", "algorithmic_bytes": b1,
                                "achieved": b1 / (res["z_all"]["ms"] * 1e-3) / 1e9,
                                "peak": hbm, "unit": "GB/s"}
    # all pairs: the I and Z slices once each beyond the environments
    # (the stacked form); FP64 flops of the stacked propagation, sum over j of
    # (rows alive) x 2 slices x chi_j chi_j+1 FMA
    b2 = 4.0 * slice_bytes
    fl2 = sum(4.0 * j * d[j] * d[j + 1] for j in range(n))
    res["zz_connected_all_pairs"]["roofline"] = {
        "bound": "hbm", "algorithmic_bytes": b2, "achieved": b2 / (res["zz_connected_all_pairs"]["ms"] * 1e-3) / 1e9,
        "peak": hbm, "unit": "GB/s", "fp64_flops": fl2,
        "fp64_tflops": fl2 / (res["zz_connected_all_pairs"]["ms"] * 1e-3) / 1e12}
    for k in ("z_all", "zz_connected_all_pairs"):
        r = res[k]["roofline"]
        r["frac"] = r["achieved"] / r["peak"] if r["peak"] else None
    return {"workload": "snake4x10_chi512 (4x10 grid on a snake path, N = 40, chi 512, seeded random MPO, "
                        "Schmidt grading exp(-%.3f r)), FP64 storage" % DECAY,
            "reps": reps, "calls": res, "clocks": clk.summary(),
            "note": "algorithmic bytes: one Pauli slice of every site = sum_p chi_p chi_p+1 x 8 B; "
                    "<Z> reads three (two environments, the Z slice), all pairs four (+ the I slice "
                    "propagated); peak = measured HBM copy bandwidth"}


def run_adjoint(args, local):
    """One gradient (checkpointed forward + backward) of sum_i zbar_i <z_i> +
    sum_{i<j} wbar_ij conn_ij on the N=24 ring (closing bond routed by swaps)
    at chi_max = 256, mixed contractions with the FP64 SVD, next to the plain
    forward steps of the same state."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2203_05871_gb300 import MIXED_TF32, Solver

    K = args.adjoint_steps
    wl = W.ring24_adjoint()
    dims, tens = W.random_mpo_state(wl.n, 256, seed=2203058712 + 2, decay=DECAY)
    stream = torch.cuda.Stream()
    s = Solver(wl.n, batch=1, chi_cap=256, stream=stream, precision=MIXED_TF32)
    s.build_gates(wl)
    rng = np.random.default_rng(2203058712)
    zb = rng.normal(size=(1, wl.n))
    wb = np.triu(rng.normal(size=(1, wl.n, wl.n)), 1)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    with ClockSampler(local) as clk:
        s.set_state(0, dims, tens)
        torch.cuda.synchronize()
        ev[0].record(stream)
        s.step(K)
        ev[1].record(stream)
        s.set_state(0, dims, tens)
        torch.cuda.synchronize()
        ev[2].record(stream)
        s.grad_forward(K)
        ev[3].record(stream)
        torch.cuda.synchronize()
        ev[4].record(stream)
        g, L = s.grad_backward(zb, wb)
        ev[5].record(stream)
        torch.cuda.synchronize()
    n_ops = s.op_counts()[0]
    st = s.status()
    s.close()
    step_ms = ev[0].elapsed_time(ev[1])
    fwd_ms = ev[2].elapsed_time(ev[3])
    bwd_ms = ev[4].elapsed_time(ev[5])
    return {"workload": "ring24_chi256 (N=24 ring, closing bond through swap gates, cutoff 1e-10, dt 0.05; "
                        "seeded random MPO start at chi 256)",
            "precision": "mixed contractions, FP64 SVD", "trotter_steps": K, "ops_per_step": n_ops,
            "s_per_step_plain": step_ms / 1e3 / K, "s_per_step_grad_forward": fwd_ms / 1e3 / K,
            "s_per_step_grad_backward": bwd_ms / 1e3 / K,
            "gradient_over_plain": (fwd_ms + bwd_ms) / step_ms if step_ms > 0 else None,
            "grad_finite": bool(np.all(np.isfinite(g))), "n_params": int(g.shape[1]),
            "loss": float(L[0]), "chi_max_seen": int(st["chi"].max()), "clocks": clk.summary()}




def arm_summary(r, world):
    """Throughput and kernel split of one timed arm."""
    prof = r["prof"]
    jac = prof["jacobi_svd"]
    steps = r["steps"]
    out = {"value": world * r["n_ops"] * steps / (r["ms"] / 1e3), "ms_per_step": r["ms"] / steps,
           "kernels": {k: {"ms_per_step": v["ms"] / steps, "launches_per_step": v["launches"] / steps}
                       for k, v in prof.items() if v["launches"]},
           "jacobi_mean_sweeps": (jac["sweeps"] / jac["svds"] if jac["svds"] else None),
           "jacobi_mean_sweeps_fp32": (jac["sweeps_fp32"] / jac["svds"] if jac["svds"] else None),
           "svd_n_effective": ((jac["flops"] / 21.0 / jac["svds"]) ** (1.0 / 3.0) if jac["svds"] else None),
           "chi_after_warmup": [int(x) for x in r["chi_warm"][0]], "clocks": r["clocks"]}
    return out


def truncation_roofline(prof, precision):
    """The truncation stage (QR + SVD, about 95% of the step) against the FP64
    peak, with the fixed algorithmic convention of 21 n^3 flops per n x n SVD."""
    jac = prof["jacobi_svd"]
    parts = ["qr", "jacobi_svd"] + (["jacobi_fp32", "precond_gemm"] if precision == "mixed" else [])
    ms = sum(prof[k]["ms"] for k in parts)
    achieved = jac["flops"] / (ms / 1e3) / 1e12 if ms > 0 else None
    names = {"qr": "qr_kernel", "jacobi_svd": "jacobi_kernel<double>", "jacobi_fp32": "jacobi_kernel<float>",
             "precond_gemm": "oz_prep/slice/gemm kernels x3 (preconditioner products)"}
    return {"kernel": "truncation stage: " + " + ".join(names[k] for k in parts),
            "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_NOMINAL_TFLOPS, "unit": "TFLOP/s",
            "frac": (achieved / FP64_PEAK_NOMINAL_TFLOPS) if achieved else None,
            "traffic": None,
            "note": "achieved = 21 n^3 flops per n x n SVD (n = 4 max(chi_l, chi_r)), the FP64 work of an ideal "
                    "Golub-Kahan SVD, over the summed CUDA-event time of the listed kernels (QR included); peak = "
                    "nominal FP64 of GB300 (2 DFMA/SM/clk x 152 SMs x 2.07 GHz; MEASURED_PEAKS.json has no "
                    "FP64 figure), of nominal; traffic: null, the stage is several kernels whose rows stay in "
                    "L2 (a jacobi_kernel<double> launch of the chain10_chi256 case read 2.8 MB of DRAM, "
                    "profiles/kernels_chain10_chi256.md)"}


def main():
    args = parse()
    if args.probe_peaks:
        return probe_peaks()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2203_05871_gb300 import build as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        B.build()
    if dist:
        dist.barrier()
    arms = ["fp64", "mixed"] if args.precision == "both" else [args.precision]
    res = {p: run_arm(args, p, world, dist, local, graph=(p == arms[-1] and not args.no_graph),
                      e2e_steps=(args.e2e_steps if p == arms[-1] else 0)) for p in arms}
    head = res["mixed"] if "mixed" in res else res["fp64"]
    hp = "mixed" if "mixed" in res else "fp64"
    wl, cap, n_ops = head["wl"], head["cap"], head["n_ops"]
    hs = arm_summary(head, world)
    e2e_value = world * n_ops * args.e2e_steps / (head["e2e_ms"] / 1e3) if args.e2e_steps > 0 else None
    prof = head["prof"]
    launches = sum(v["launches"] for v in prof.values())      # kernels, as counted by the library
    dtype = (("mixed: tcgen05 %s slice products (six 8-bit slices, exact level sums, fp64 re-accumulated) for the "
              "contractions and preconditioner GEMMs, fp32-preconditioned fp64 QR + Jacobi SVD" % args.mixed_kind)
             if hp == "mixed" else "f64")
    line = {
        "metric": "gate_applications_per_sec", "value": hs["value"], "unit": "gate-applications/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": hs["ms_per_step"],
        "s_per_trotter_step": hs["ms_per_step"] / 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic",
        "config": {"workload": args.workload, "n_qubits": wl.n, "batch": wl.batch, "chi_max": cap,
                   "cutoff": float(wl.cutoff[0]),
                   "dt": wl.dt, "ops_per_step": n_ops, "swaps_per_step": head["n_swaps"], "precision": hp,
                   "qr": "blocked" if (hp == "mixed" and args.qr_blocked) else "column",
                   "parallelism": f"replicas{world}", "l2": "flushed (256 MB write) between timed steps",
                   "start": "seeded random MPO at chi_max, Schmidt grading exp(-%.3f r)" % (
                       DECAY if "flat" not in args.workload else 0.0)},
        "e2e": {"value": e2e_value, "unit": "gate-applications/s", "h2d_bytes_per_step": head["flat_bytes"],
                "d2h_bytes_per_step": wl.n * wl.batch * 8},
        "gpu_launches": launches,
        "kernels": hs["kernels"],
        "jacobi_mean_sweeps": hs["jacobi_mean_sweeps"],
        "jacobi_mean_sweeps_fp32": hs["jacobi_mean_sweeps_fp32"],
        "svd_n_effective": hs["svd_n_effective"],
        "chi_after_warmup": hs["chi_after_warmup"],
        "jacobi_critical_sweeps": ([prof["jacobi_svd"]["critical_sweeps"] / prof["jacobi_svd"]["chunks"],
                                    prof["jacobi_svd"]["critical_sweeps_fp32"] / prof["jacobi_svd"]["chunks"]]
                                   if prof["jacobi_svd"].get("chunks") else None),
        "roofline": truncation_roofline(prof, hp),
        "roofline_contraction": contraction_roofline(prof, args.mixed_kind) if hp == "mixed" else None,
        "roofline_qr": qr_roofline(prof),
        "autotune": {"jacobi_rows_per_block": head["tuned"],
                     "note": "(chi_l x chi_r): [FP64 pass, FP32 pass], measured before the timed steps"},
        "graph_step": ({"ms_per_step": head["graph_ms"] / args.steps,
                        "note": "same steps replayed from one captured CUDA graph (device-side planning)"}
                       if head["graph_ms"] is not None else None),
        "clocks": head["clocks"],
        "status": int(head["status"]["status"][0]), "chi_max_seen": int(head["status"]["chi"].max()),
    }
    if "fp64" in res and hp != "fp64":
        f = arm_summary(res["fp64"], world)
        f["dtype"] = "f64"
        f["note"] = "the same workload, steps and start on the FP64 path (FP64 contractions, FP64 QR + Jacobi)"
        line["fp64_path"] = f
        line["speedup_mixed_vs_fp64"] = res["fp64"]["ms"] / res["fp64"]["steps"] / hs["ms_per_step"]
    if args.per_gate_steps > 0:
        g = run_arm(args, "fp64", world, dist, local, steps=args.per_gate_steps, warmup=1, max_slots=1,
                    graph=False, e2e_steps=0)
        pg = arm_summary(g, world)
        pg["note"] = ("FP64 path with one two-site op in flight (max_slots = 1): the plain per-gate path; "
                      "1 warm-up step, %d timed" % args.per_gate_steps)
        line["fp64_per_gate"] = pg
        line["speedup_mixed_vs_fp64_per_gate"] = pg["ms_per_step"] / hs["ms_per_step"]
    if args.batched_steps > 0 and args.workload != "batch64_chain16":
        bt = run_arm(args, hp, world, dist, local, workload="batch64_chain16", steps=args.batched_steps, warmup=1,
                     graph=False, e2e_steps=0)
        bs = arm_summary(bt, world)
        bs.pop("chi_after_warmup", None)
        bs["note"] = ("64 independent N=16 chains, chi_max from {32, 64, 128, 256} per instance, each started "
                      "at its saturated chi; %s path, 1 warm-up step, %d timed" % (hp, args.batched_steps))
        bs["ops_per_step"] = bt["n_ops"]
        line["batched"] = bs
    if args.adjoint_steps > 0:
        line["adjoint"] = run_adjoint(args, local)
    if not args.no_observables:
        try:
            line["observables"] = run_observables(args, local)
        except Exception as exc:   # keep the headline line; report what failed
            line["observables"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_subprocess(args, "lapack", args.cpu_ops, 1)
        if not args.no_cpu_plain:
            line["cpu_baseline_plain"] = cpu_baseline_subprocess(args, "jacobi", 1, 0)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
