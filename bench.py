"""Benchmark of the block saddle-point operator and MINRES on one GB300.

Headline (`value`): GDOF/s of the fused FP64 block-operator apply
y = AA x (RT mass + D + D^T + W^-1, Eq. transformed-saddle-point) at k = 4 on a
64^3 perturbed hex mesh (67,305,472 DOFs); one step = one apply. Also reported:
the element kernel's roofline (FP64 ALU bound), the same apply through the C ABI
with host buffers (e2e), an FP64 MINRES time-to-solution on the same problem,
clocks sampled during the timed region, and the CPU oracle on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload
(weak scaling, no data-path collective); the timing is the max over ranks.
"""
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

import synth  # noqa: E402

METRIC = "GDOF/s of block operator apply at p=4; MINRES time-to-1e-8 resid, mixed/learned vs FP64"
# workload: grad-div on the unit cube, 64^3 elements, interior vertices moved by
# U(-0.15 h, 0.15 h), k = 4 (RT_4 x Q_3), q = 6, alpha = 1, beta = exp(2 Z) per
# element, u.n = 0 on all six sides
NX, K, Q, PERTURB, SIGMA, ESS, SEED = 64, 4, 6, 0.15, 2.0, 63, 2304
# measured FP64 FMA rate of this GPU model: 152 SMs x 2 FP64 FMA lanes/clk x 2 flops
FP64_PEAK_GFLOPS_AT_MAX_CLOCK = 152 * 2 * 2 * 2.070
# probed double-float FMA rate of this GPU model (FP32 pairs on the FP32 pipe), 2 flops each
DF_PEAK_FP64_EQUIV_GFLOPS = 2 * 2471.0
# DRAM bytes (read + write) per element of the element kernel, from one ncu capture of the 24^3
# case of the same recipe (13,824 elements); to be dropped when the kernel changes
ELEM_TRAFFIC_BYTES_PER_ELEMENT = {(4, 6, "f64"): 673.985024e6 / 13824,   # FP64 kernel
                                  (4, 6, "df"): 674.329088e6 / 13824}    # double-float kernel


def _measured_hbm_gbs(default=6792.4):
    """HBM copy bandwidth (read + write bytes) measured on this GPU pool, from
    MEASURED_PEAKS.json beside this file when present; else the value it held when
    these kernels were measured."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v if v > 0 else default
    except (OSError, ValueError, KeyError, TypeError):
        return default


HBM_GBS_MEASURED = _measured_hbm_gbs()


def workload(n=NX):
    vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=PERTURB, seed=SEED)
    E = n ** 3
    alpha = np.ones(E)
    beta = synth.lognormal(E, SIGMA, seed=SEED + 1)
    return vx, vy, vz, alpha, beta


def elem_flops(k, q):
    """Algorithmic FP64 flops of the fused element kernel per element: sum-factorised
    interpolation of the three RT components to the q^3 points and its transpose,
    the symmetric 3x3 geometric factor at each point, the dense k^3 x k^3 W_e^-1
    product, the cell divergences and the own-cell D^T terms (an FMA = 2 flops)."""
    K, Q = k, q
    interp = (K * K * Q * (K + 1) + Q * K * Q * K + Q * Q * Q * K            # x component
              + (K + 1) * K * Q * K + Q * K * Q * (K + 1) + Q * Q * Q * K    # y component
              + K * (K + 1) * Q * K + Q * (K + 1) * Q * K + Q * Q * Q * (K + 1))  # z component
    macs = 2 * interp + 9 * Q ** 3 + K ** 6
    nrt = 3 * (K + 1) * K * K
    return 2 * macs + 6 * K ** 3 + 3 * nrt + K ** 3


def elem_flops_affine(k, q):
    """The same count for the affine fast path: the geometric factor is one 3x3 matrix per
    element scaled by w_p (the weight product and three scalings per point), and W_e^-1 is
    det J (H^-1 x H^-1 x H^-1), three k x k contractions (3 k^4 MACs) and one scaling."""
    K, Q = k, q
    interp = (K * K * Q * (K + 1) + Q * K * Q * K + Q * Q * Q * K
              + (K + 1) * K * Q * K + Q * K * Q * (K + 1) + Q * Q * Q * K
              + K * (K + 1) * Q * K + Q * (K + 1) * Q * K + Q * Q * Q * (K + 1))
    macs = 2 * interp + 9 * Q ** 3 + 3 * K ** 4
    nrt = 3 * (K + 1) * K * K
    return 2 * macs + 5 * Q ** 3 + K ** 3 + 6 * K ** 3 + 3 * nrt + K ** 3


def elem_bytes_affine(n_elem, n_rt, n_l2):
    """Algorithmic DRAM bytes of one affine fast-path apply: read x, write y and 8
    doubles per element (the constant geometric factor and det J)."""
    return 8 * (2 * (n_rt + n_l2) + 8 * n_elem)


def alg_bytes(n_rt, n_l2, n_vert, n_elem, q=None):
    """Algorithmic DRAM bytes of one FP64 block apply (the method's own traffic): read x and
    write y (8 (2 N_RT + 2 N_L2)), the vertex coordinates (24 per vertex) and two coefficients
    per element (16). q given: the variant that keeps the geometric factors per quadrature
    point (7 doubles per point: the 6 entries of J^T J/det J and w/det J), 56 q^3 per element."""
    b = 8 * (2 * n_rt + 2 * n_l2) + 24 * n_vert + 16 * n_elem
    return b + (56 * q ** 3 * n_elem if q else 0)


def roofline(op, nx, kern_ms, emulated):
    """Roofline object of the fused element kernel against HBM on the method's algorithmic
    bytes (the per-point variant: this kernel reads stored geometric factors), with the
    bytes the kernel streams by its storage choices (per-point factors and the dense
    per-element W^-1, 8 (2N + E (6 q^3 + k^6 + 1))) beside them. The kernel is bound by
    arithmetic issue, not by HBM: the "alu" object gives its double-float (or FP64)
    arithmetic rate against the probed peak of that arithmetic."""
    nv = (nx + 1) ** 3
    abytes = alg_bytes(op.n_rt, op.n_l2, nv, op.n_elem, Q)
    sbytes = elem_bytes(K, Q, op.n_elem, op.n_rt, op.n_l2)
    key = (K, Q, "df" if emulated else "f64")
    traffic = ELEM_TRAFFIC_BYTES_PER_ELEMENT[key] * op.n_elem if key in ELEM_TRAFFIC_BYTES_PER_ELEMENT else None
    gbs = abytes / (kern_ms * 1e-3) / 1e9
    flops = elem_flops(K, Q) * op.n_elem
    gflops = flops / (kern_ms * 1e-3) / 1e9
    if emulated:
        alu = {"arithmetic": "double-float (FP32 pairs) on the FP32 pipe", "achieved": gflops,
               "peak": DF_PEAK_FP64_EQUIV_GFLOPS, "unit": "GFLOP/s (FP64-equivalent)",
               "frac": gflops / DF_PEAK_FP64_EQUIV_GFLOPS,
               "peak_source": "probe: 2471 G double-float FMA/s on this GPU model (2 flops each)"}
    else:
        alu = {"arithmetic": "FP64", "achieved": gflops, "peak": FP64_PEAK_GFLOPS_AT_MAX_CLOCK, "unit": "GFLOP/s",
               "frac": gflops / FP64_PEAK_GFLOPS_AT_MAX_CLOCK,
               "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz (probe: 1189 GFLOP/s at 2002 MHz)"}
    return {"bound": "hbm", "achieved": gbs, "peak": HBM_GBS_MEASURED, "unit": "GB/s",
            "frac": gbs / HBM_GBS_MEASURED, "traffic": traffic,
            "traffic_over_algorithmic": traffic / abytes if traffic else None,
            "kernel": "k_elem_op<%s,double,%d,%d,8>" % ("dfloat" if emulated else "double", K, Q),
            "kernel_ms": kern_ms, "algorithmic_bytes_per_launch": abytes,
            "algorithmic_bytes": "8(2 N_RT + 2 N_L2) + 24 N_vert + 16 E + 56 q^3 E (per-point geometric factors)",
            "streamed_bytes_per_launch": sbytes,
            "streamed_bytes": "8 (2 N + E (6 q^3 + k^6 + 1)): per-point factors and the stored dense W_e^-1",
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)", "flops_per_launch": flops, "alu": alu}


def elem_bytes(k, q, n_elem, n_rt, n_l2):
    """Bytes the fused element kernel streams by its storage choices: read x (u, q),
    write y (u, q), the geometric factors (6 q^3 doubles per element), W_e^-1 (k^6
    doubles) and the coefficient scale."""
    return 8 * (2 * (n_rt + n_l2) + n_elem * (6 * q ** 3 + k ** 6 + 1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


_ORACLE = {}


def _oracle_worker(arg):
    """One process of the CPU baseline: builds the oracle on an n^3-element mesh of the
    metric recipe (once per process) and repeats its assembled-CSR block apply for about
    `seconds` (scipy's SpMV runs on one thread). Returns (DOFs applied, seconds, DOFs
    per apply)."""
    seconds, n = arg
    if n not in _ORACLE:
        from oracle.assembly import GRAD_DIV, Problem
        vx, vy, vz, alpha, beta = workload(n)
        prob = Problem(n, n, n, K, vx, vy, vz, alpha, beta, kind=GRAD_DIV, ess_mask=ESS, q=Q)
        x = synth.uniform(prob.n, seed=SEED)
        prob.apply_op(x)
        _ORACLE[n] = (prob, x)
    prob, x = _ORACLE[n]
    reps, t0 = 0, time.perf_counter()
    while True:
        prob.apply_op(x)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return prob.n * reps, el, prob.n


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


class OraclePool:
    """`procs` single-threaded processes (spawned, not forked) that each hold their own copy
    of the CPU oracle on an n^3-element sample of the metric workload."""

    def __init__(self, procs, n=4):
        import multiprocessing as mp
        self.procs, self.n = procs, n
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(procs)
        finally:
            for v, old in saved.items():
                if old is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old
        self.pool.map(_oracle_worker, [(0.0, n)] * procs)  # build the samples

    def run(self, seconds):
        """Every process applies its oracle for about `seconds`. Returns GDOF/s summed over
        the processes (over the slowest process's time), that time and DOFs per apply."""
        res = self.pool.map(_oracle_worker, [(seconds, self.n)] * self.procs)
        el = max(r[1] for r in res)
        return sum(r[0] for r in res) / el / 1e9, el, res[0][2]

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(seconds=8.0):
    """cpu_baseline object: the oracle on every host core (os.cpu_count() processes) and
    on one core, on a 4^3-element sample of the metric workload."""
    cores = os.cpu_count() or 1
    one = OraclePool(1)
    v1, el1, ndof = one.run(seconds)
    one.close()
    every = OraclePool(cores)
    vall, elall, _ = every.run(seconds)
    every.close()
    return {"value": vall, "unit": "GDOF/s", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": ("4^3 elements of the metric recipe (%d DOFs): assembled-CSR block applies (scipy SpMV, one "
                       "thread per process) for %.1f s in each of %d spawned processes, one per host core"
                       % (ndof, elall, cores)),
            "single_core": {"value": v1, "unit": "GDOF/s", "cores": 1, "seconds": el1}}


def native_apply(args, nx, vx, vy, vz, alpha, beta, stream):
    """The same apply with the FP64 element kernel (separate handle), for comparison."""
    import torch
    import paper_2304_12387_gb300 as hd
    op = hd.Operator(nx, nx, nx, K, vx, vy, vz, alpha, beta, kind=hd.HD_GRAD_DIV, ess_mask=ESS, q=Q,
                     cycle=args.cycle, fp64_emulation=0, stream=stream)
    x = torch.from_numpy(synth.uniform(op.n, seed=SEED)).cuda()
    y = torch.empty_like(x)
    for _ in range(3):
        op.hd_apply_op(x, y)
    steps = max(5, args.steps // 10)
    op.hd_profile(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        op.hd_apply_op(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    op.hd_profile(0)
    launches, kms = op.hd_profile_read()
    ms = e0.elapsed_time(e1) / steps
    r = {"value": op.n / (ms * 1e-3) / 1e9, "unit": "GDOF/s", "ms_per_step": ms, "steps": steps,
         "roofline": roofline(op, nx, kms / max(1, launches), False)}
    op.close()
    return r


def f32_apply(args, op, nx):
    """The FP32 operator of the mixed-precision solves (FP32 element kernel, FP32 vectors),
    on the main line's handle: GDOF/s and its HBM roofline. Algorithmic bytes per apply:
    4 (2N + E (6 q^3 + k^6 + 1)) (FP32 vectors in and out, FP32 G, W_e^-1 and c_e)."""
    import torch
    n = op.n
    x = torch.from_numpy(synth.uniform(n, seed=SEED)).float().cuda()
    y = torch.empty_like(x)
    for _ in range(3):
        op.hd_apply_op_f32(x, y)
    steps = max(5, args.steps // 10)
    op.hd_profile(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        op.hd_apply_op_f32(x, y)
    e1.record()
    torch.cuda.synchronize()
    op.hd_profile(0)
    launches, kms = op.hd_profile_read()
    kms = kms / max(1, launches)
    E = nx ** 3
    alg = alg_bytes(op.n_rt, op.n_l2, (nx + 1) ** 3, E, Q) // 2   # the same counts in FP32
    streamed = 4 * (2 * n + E * (6 * Q ** 3 + K ** 6 + 1))
    peak = _measured_hbm_gbs()
    return {"value": n / (e0.elapsed_time(e1) / steps * 1e-3) / 1e9, "unit": "GDOF/s",
            "ms_per_step": e0.elapsed_time(e1) / steps, "steps": steps, "kernel_ms": kms,
            "algorithmic_bytes_per_launch": alg, "hbm_frac_of_measured": alg / (kms * 1e-3) / 1e9 / peak,
            "streamed_bytes_per_launch": streamed,
            "streamed_hbm_frac_of_measured": streamed / (kms * 1e-3) / 1e9 / peak}


def affine_apply(args, stream):
    """Metric 1 on the Cartesian geometry (M64-affine): the unperturbed mesh of the
    same size and coefficients, q = k + 1, the same element kernel and precision as
    the main line; a separate handle."""
    import torch
    import paper_2304_12387_gb300 as hd
    nx = args.n
    vx, vy, vz = synth.lattice_vertices(nx, nx, nx)
    _, _, _, alpha, beta = workload(nx)
    q = K + 1
    op = hd.Operator(nx, nx, nx, K, vx, vy, vz, alpha, beta, kind=hd.HD_GRAD_DIV, ess_mask=ESS, q=q, affine=True,
                     cycle=args.cycle, fp64_emulation=int(args.fp64_emulation), stream=stream)
    x = torch.from_numpy(synth.uniform(op.n, seed=SEED)).cuda()
    y = torch.empty_like(x)
    for _ in range(3):
        op.hd_apply_op(x, y)
    steps = max(5, args.steps // 10)
    op.hd_profile(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        op.hd_apply_op(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    op.hd_profile(0)
    launches, kms = op.hd_profile_read()
    ms = e0.elapsed_time(e1) / steps
    kern_ms = kms / max(1, launches)
    abytes = alg_bytes(op.n_rt, op.n_l2, (nx + 1) ** 3, op.n_elem)
    sbytes = elem_bytes_affine(op.n_elem, op.n_rt, op.n_l2)
    flops = elem_flops_affine(K, q) * op.n_elem
    # the same operator on the tensor cores (FP16-pair operands, FP32 accumulation): the inner
    # operator of the mixed-precision solves on affine meshes, FP64 and FP32 vectors
    tc = {}
    for key, xx, yy, fn in (("f64_vectors", x, y, op.hd_apply_op_tc),
                            ("f32_vectors", x.float(), y.float(), op.hd_apply_op_tc_f32)):
        for _ in range(3):
            fn(xx, yy)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            fn(xx, yy)
        t1.record(stream)
        torch.cuda.synchronize()
        tms = t0.elapsed_time(t1) / steps
        ab = abytes if key == "f64_vectors" else abytes // 2
        tc[key] = {"value": op.n / (tms * 1e-3) / 1e9, "unit": "GDOF/s", "ms_per_step": tms,
                   "hbm_frac_of_measured": ab / (tms * 1e-3) / 1e9 / HBM_GBS_MEASURED}
    ref = torch.empty_like(x)
    op.hd_apply_op(x, ref)
    op.hd_apply_op_tc(x, y)
    torch.cuda.synchronize()
    tc["max_rel_diff_vs_fp64_apply"] = float((y - ref).abs().max() / ref.abs().max())
    tc["status"] = int(op.hd_tc_status())
    tc["kernel"] = "k_op_tc<double|float,%d>: tcgen05.mma kind::f16, FP16 pairs, FP32 accumulators in TMEM" % K
    r = {"workload": "M%d-affine: the same recipe on the unperturbed mesh, q=%d" % (nx, q),
         "value": op.n / (ms * 1e-3) / 1e9, "unit": "GDOF/s", "ms_per_step": ms, "steps": steps,
         "kernel": "k_elem_op<%s,double,%d,%d,8,affine>" % ("dfloat" if args.fp64_emulation else "double", K, q),
         "kernel_ms": kern_ms, "algorithmic_bytes_per_launch": abytes, "streamed_bytes_per_launch": sbytes,
         "element_data": "affine fast path: 64 B per element (constant geometric factor, det J)",
         "hbm_frac_of_measured": abytes / (kern_ms * 1e-3) / 1e9 / HBM_GBS_MEASURED,
         "fp64_equivalent_gflops": flops / (kern_ms * 1e-3) / 1e9, "tensor_core_apply": tc}
    op.close()
    return r


def affine_workload(name):
    """The affine solve workloads: C4, grad-div on the unit cube, 48^3 elements, k = 4, a
    seeded bent tube (radius 0.15) with alpha = 1e3, beta = 1 inside and alpha = 1,
    beta = 1e-3 outside, u.n = 0; C3, Darcy on [0,1200]x[0,2200]x[0,170] with 60x220x85
    elements, k = 2, gamma = 0, eps = exp(3Z) per layer (AR(1) along x, correlation length
    10 cells), u.n = 0 everywhere (pure Neumann: the q block is singular, projected)."""
    import paper_2304_12387_gb300 as hd
    if name == "C4":
        n = 48
        vx, vy, vz = synth.lattice_vertices(n, n, n)
        inside = synth.bent_tube_mask(n, n, n, seed=SEED)
        return dict(dims=(n, n, n), k=4, kind=hd.HD_GRAD_DIV, v=(vx, vy, vz), c0=np.where(inside, 1e3, 1.0),
                    c1=np.where(inside, 1.0, 1e-3))
    nx, ny, nz = 60, 220, 85
    vx, vy, vz = synth.lattice_vertices(nx, ny, nz, extent=(1200.0, 2200.0, 170.0))
    eps = synth.layered_permeability(nx, ny, nz, sigma=3.0, corr_len=10.0, seed=SEED)
    return dict(dims=(nx, ny, nz), k=2, kind=hd.HD_DARCY, v=(vx, vy, vz), c0=eps, c1=np.zeros(nx * ny * nz))


def affine_solves(args, stream):
    """Time to a true relative residual of 1e-8 on the affine workloads (C4, C3): FP64 MINRES
    (double-float element kernel, FP64 V/W-cycle), mixed-precision MINRES with the FP32
    CUDA-core inner operator, the same with the tensor-core inner operator, and mixed GMRES
    (block-triangular) with the tensor-core inner operator; the error of each solution
    against the FP64 one. Setup is timed separately."""
    import torch
    import paper_2304_12387_gb300 as hd
    out = {}
    for name in ("C4", "C3"):
        w = affine_workload(name)
        nx, ny, nz = w["dims"]
        t0 = time.perf_counter()
        op = hd.Operator(nx, ny, nz, w["k"], *w["v"], w["c0"], w["c1"], kind=w["kind"], ess_mask=ESS,
                         q=w["k"] + 1, affine=True, cycle=2, smooth_levels=2, fp64_emulation=1, stream=stream)
        torch.cuda.synchronize()
        r = {"dofs": op.n, "elements": op.n_elem, "k": w["k"], "setup_s": time.perf_counter() - t0}
        b = torch.from_numpy(synth.uniform(op.n, seed=SEED + 7)).cuda()
        b[torch.from_numpy(op.hd_get_ess_dofs()).cuda()] = 0.0
        if name == "C3":
            b[op.n_rt:] -= b[op.n_rt:].mean()  # compatible right-hand side of the singular problem
        sols = {}

        def rec(key, st, info, xs):
            sols[key] = xs
            r[key] = {"status": int(st), "iterations": info["iterations"], "outer": info.get("outer", info.get("cycles")),
                      "ms": info["ms_total"], "true_relres": info["true_relres"]}
            if key != "minres_fp64":
                ref = sols["minres_fp64"]
                r[key]["rel_diff_vs_fp64_solution"] = float(torch.linalg.vector_norm(xs - ref) /
                                                             torch.linalg.vector_norm(ref))
                r[key]["speedup_vs_minres_fp64"] = r["minres_fp64"]["ms"] / max(info["ms_total"], 1e-9)

        xs = torch.zeros_like(b)
        st, info = op.hd_minres_solve(b, xs, rtol=1e-8, maxit=args.solve_maxit, check_every=16, outer_rtol=1e-8,
                                      max_outer=40)
        rec("minres_fp64", st, info, xs)
        for key, mode in (("minres_mixed", 0), ("minres_mixed_tc", 1)):
            op.hd_set_inner_operator(mode)
            xs = torch.zeros_like(b)
            st, info = op.hd_minres_solve(b, xs, rtol=args.inner_rtol, maxit=args.solve_maxit, check_every=16,
                                          precision=1, outer_rtol=1e-8, max_outer=40)
            rec(key, st, info, xs)
        op.hd_set_inner_operator(1)
        xs = torch.zeros_like(b)
        st, info = op.hd_gmres_solve(b, xs, rtol=1e-8, maxit=args.solve_maxit, restart=args.gmres_restart,
                                     prec=hd.HD_GMRES_BLOCK_TRI, precision=1, inner_rtol=args.gmres_inner_rtol)
        rec("gmres_tri_mixed_tc", st, info, xs)
        r["tc_status"] = int(op.hd_tc_status())
        op.close()
        out[name] = r
    return out


def max_over_ranks(value, dist):
    """Largest value over the ranks (a job takes as long as its slowest rank);
    the value itself without a process group."""
    if dist is None:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank, world):
    """The oracle arm: W warm-up and K timed steps on every host core, each step a
    bounded sample of the metric workload (every core applies the assembled-CSR block
    operator of its own copy of a 4^3-element mesh of the same recipe for a fixed
    time, sized so that the whole run takes about a minute at most)."""
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    steps, warmup = max(1, args.steps), max(0, args.warmup)
    step_s = min(2.0, 60.0 / (steps + warmup))
    pool = OraclePool(cores)
    for _ in range(warmup):
        pool.run(step_s)
    vals, els, ndof = [], [], 0
    for _ in range(steps):
        v, el, ndof = pool.run(step_s)
        vals.append(v)
        els.append(el)
    pool.close()
    gdofs = statistics.median(vals)
    sample = ("4^3 elements of the 64^3 recipe (%d DOFs); a step = %.2f s of assembled-CSR block applies in "
              "each of %d spawned single-threaded processes (one per host core)" % (ndof, step_s, cores))
    line = {"impl": "reference", "metric": METRIC, "value": gdofs, "unit": "GDOF/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warmup, "ms_per_step": statistics.median(els) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "M64-perturbed recipe on a 4^3-element sample per core (k=4, q=6, %d DOFs)" % ndof},
            "cpu_baseline": {"value": gdofs, "unit": "GDOF/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": gdofs, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, dist):
    import torch
    import paper_2304_12387_gb300 as hd
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    nx = args.n
    vx, vy, vz, alpha, beta = workload(nx)
    t0 = time.perf_counter()
    op = hd.Operator(nx, nx, nx, K, vx, vy, vz, alpha, beta, kind=hd.HD_GRAD_DIV, ess_mask=ESS, q=Q,
                     cycle=args.cycle, fp64_emulation=int(args.fp64_emulation),
                     smooth_levels=args.smooth_levels, w_levels=args.w_levels, stream=stream)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    n = op.n
    x = torch.from_numpy(synth.uniform(n, seed=SEED)).cuda()
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        op.hd_apply_op(x, y)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        op.hd_profile(1)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            op.hd_apply_op(x, y)
        ev1.record(stream)
        torch.cuda.synchronize()
        op.hd_profile(0)
    if dist:
        dist.barrier()
    ms_total = ev0.elapsed_time(ev1)
    launches, kern_ms = op.hd_profile_read()
    ms_total = max_over_ranks(ms_total, dist)
    ms_step = ms_total / args.steps
    value = world * n / (ms_step * 1e-3) / 1e9
    # roofline of the fused element kernel (one launch per apply)
    kern_avg_ms = kern_ms / max(1, launches)
    clocks = clk.summary()
    roof = roofline(op, nx, kern_avg_ms, bool(args.fp64_emulation))
    # e2e: the same apply through the C ABI with pinned host buffers, copies inside the region
    xh = torch.from_numpy(synth.uniform(n, seed=SEED)).pin_memory()
    yh = torch.empty(n, dtype=torch.float64).pin_memory()
    op.hd_apply_op_host(xh, yh)
    e2e_steps = max(3, args.steps // 10)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        op.hd_apply_op_host(xh, yh)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist)
    e2e = {"value": world * n / e2e_s / 1e9, "unit": "GDOF/s", "h2d_bytes_per_step": 8 * n,
           "d2h_bytes_per_step": 8 * n, "ms_per_step": e2e_s * 1e3}
    out = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32x2" if args.fp64_emulation else "f64", "data": "synthetic",
           "config": {"workload": ("M64-perturbed" if nx == NX else "M%d-perturbed (profiling size)" % nx)
                                  + ": grad-div, %d^3 hex elements of the unit cube with interior " % nx +
                                  "vertices moved by U(-0.15h,0.15h) (seed 2304), RT_4 x Q_3 (k=4), q=6, "
                                  "alpha=1, beta=exp(2Z) per element, u.n=0 on all sides",
                      "dofs": n, "n_rt": op.n_rt, "n_l2": op.n_l2, "elements": op.n_elem,
                      "step": "one fused block-operator apply (hd_apply_op), FP64 vectors in and out; element "
                              "kernel in " + ("double-float (FP32 pairs, FP64 parity 1e-12 in the tests)"
                                              if args.fp64_emulation else "FP64"),
                      "l2": "inputs larger than L2 (x, y: 538 MB each; W^-1 8.6 GB; geometric factors 2.7 GB)",
                      "winv": "dense per-element inverse", "setup_s": setup_s,
                      "schur_cycle": ("W" if args.cycle == 2 else "V") +
                                     {0: ", plain aggregation", 1: ", smoothed aggregation on the first level",
                                      2: ", smoothed aggregation on the first two levels"}[args.smooth_levels]},
           "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
    out["apply_fp32_inner"] = f32_apply(args, op, nx)
    if args.fp64_emulation and not args.no_native:
        out["apply_native_fp64"] = native_apply(args, nx, vx, vy, vz, alpha, beta, stream)
    if not args.no_affine:
        out["apply_affine"] = affine_apply(args, stream)
    if not args.no_solve and not args.no_affine:
        out["affine_solves"] = affine_solves(args, stream)
    if not args.no_solve and not args.no_learned:
        out["minres_learned"] = learned_study(args, stream)
    # MINRES time to a true relative residual of 1e-8 on the same problem: FP64, and
    # mixed precision (FP32 operator and V-cycle inside an FP64 residual correction)
    if not args.no_solve:
        b = torch.from_numpy(synth.uniform(n, seed=SEED + 7)).cuda()
        ess = torch.from_numpy(op.hd_get_ess_dofs()).cuda()
        b[ess] = 0.0
        sols = {}
        solvers = set(args.solvers.split(","))
        for key, prec, rtol in (("minres_fp64", 0, 1e-8), ("minres_mixed", 1, args.inner_rtol)):
            if "minres" not in solvers:
                break
            xs = torch.zeros_like(b)
            st, info = op.hd_minres_solve(b, xs, rtol=rtol, maxit=args.solve_maxit, check_every=16,
                                          precision=prec, outer_rtol=1e-8, max_outer=40)
            sols[key] = xs
            out[key] = {"status": int(st), "iterations": info["iterations"], "outer": info["outer"],
                        "ms": info["ms_total"], "true_relres": info["true_relres"], "inner_rtol": rtol,
                        "ms_per_iteration": info["ms_total"] / max(1, info["iterations"])}
        if "minres" in solvers:
            d = float(torch.linalg.vector_norm(sols["minres_mixed"] - sols["minres_fp64"]) /
                      torch.linalg.vector_norm(sols["minres_fp64"]))
            out["minres_mixed"]["rel_diff_vs_fp64_solution"] = d
            out["minres_mixed"]["speedup_vs_fp64"] = out["minres_fp64"]["ms"] / out["minres_mixed"]["ms"]
        def vs_minres(xs, ms):
            if "minres_fp64" not in sols:
                return {}
            ref = sols["minres_fp64"]
            return {"rel_diff_vs_minres_fp64_solution": float(torch.linalg.vector_norm(xs - ref) /
                                                              torch.linalg.vector_norm(ref)),
                    "speedup_vs_minres_fp64": out["minres_fp64"]["ms"] / ms}

        if "gmres" in solvers:
            # GMRES with the block upper-triangular preconditioner (the remark in Sec. 2.3), FP64,
            # to the same true relative residual
            xs = torch.zeros_like(b)
            st, info = op.hd_gmres_solve(b, xs, rtol=1e-8, maxit=args.solve_maxit, restart=args.gmres_restart,
                                         prec=hd.HD_GMRES_BLOCK_TRI)
            out["gmres_tri_fp64"] = {
                "status": int(st), "iterations": info["iterations"], "restart": args.gmres_restart,
                "cycles": info["cycles"], "ms": info["ms_total"], "true_relres": info["true_relres"],
                "ms_per_iteration": info["ms_total"] / max(1, info["iterations"]),
                **vs_minres(xs, info["ms_total"])}
            # the same with every cycle in FP32 (basis, Gram-Schmidt, operator, V-cycle) and the FP64
            # residual at every restart
            xs = torch.zeros_like(b)
            st, info = op.hd_gmres_solve(b, xs, rtol=1e-8, maxit=args.solve_maxit, restart=args.gmres_restart,
                                         prec=hd.HD_GMRES_BLOCK_TRI, precision=1, inner_rtol=args.gmres_inner_rtol)
            out["gmres_tri_mixed"] = {
                "status": int(st), "iterations": info["iterations"], "restart": args.gmres_restart,
                "inner_rtol": args.gmres_inner_rtol, "cycles": info["cycles"], "ms": info["ms_total"],
                "true_relres": info["true_relres"], "ms_per_iteration": info["ms_total"] / max(1, info["iterations"]),
                **vs_minres(xs, info["ms_total"])}
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(seconds=8.0)
    op.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_iterations(args):
    """Mesh and degree (in)dependence of the iteration counts (Metric 2's study): FP64
    MINRES to a true relative residual of 1e-8 on the metric recipe (perturbed mesh,
    beta = exp(2Z), u.n = 0, q = k + 2) at several element counts and degrees, with
    the plain-aggregation W-cycle and the smoothed-aggregation W-cycles with one and
    with two smoothed levels; mixed precision beside FP64 for the last. For odd k also
    the element-aligned aggregates (plain and one smoothed level, FP64 and mixed)."""
    import torch
    import paper_2304_12387_gb300 as hd
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    stream = torch.cuda.current_stream()
    cases = [(16, 4), (32, 4), (64, 4), (96, 4), (32, 2), (32, 3), (32, 5)]
    rows = []
    for nx, k in cases:
        vx, vy, vz, alpha, beta = workload(nx)
        row = {"elements": nx, "k": k}
        variants = [("plain", 0, 0), ("smoothed1", 1, 0), ("smoothed2", 2, 0)]
        if k % 2:  # element-aligned aggregates (the pairs straddle element boundaries for odd k)
            variants += [("aligned_plain", 0, 1), ("aligned_smoothed1", 1, 1)]
        for name, sl, agg in variants:
            op = hd.Operator(nx, nx, nx, k, vx, vy, vz, alpha, beta, kind=hd.HD_GRAD_DIV, ess_mask=ESS, q=k + 2,
                             cycle=2, fp64_emulation=1, smooth_levels=sl, aggregation=agg, stream=stream)
            row["dofs"] = op.n
            b = torch.from_numpy(synth.uniform(op.n, seed=SEED + 7)).cuda()
            b[torch.from_numpy(op.hd_get_ess_dofs()).cuda()] = 0.0
            if sl == 2 and not agg:
                x = torch.zeros_like(b)
                st, info = op.hd_gmres_solve(b, x, rtol=1e-8, maxit=args.solve_maxit, restart=args.gmres_restart,
                                             prec=hd.HD_GMRES_BLOCK_TRI)
                row["gmres_tri"] = {"status": int(st), "iterations": info["iterations"], "cycles": info["cycles"],
                                    "ms": round(info["ms_total"], 1), "true_relres": info["true_relres"]}
                x = torch.zeros_like(b)
                st, info = op.hd_gmres_solve(b, x, rtol=1e-8, maxit=args.solve_maxit, restart=args.gmres_restart,
                                             prec=hd.HD_GMRES_BLOCK_TRI, precision=1,
                                             inner_rtol=args.gmres_inner_rtol)
                row["gmres_tri_mixed"] = {"status": int(st), "iterations": info["iterations"],
                                          "cycles": info["cycles"], "ms": round(info["ms_total"], 1),
                                          "true_relres": info["true_relres"]}
            for prec in ((0, 1) if sl == 2 or (agg and sl == 1) else (0,)):
                x = torch.zeros_like(b)
                st, info = op.hd_minres_solve(b, x, rtol=1e-4 if prec else 1e-8, maxit=args.solve_maxit,
                                              check_every=16, precision=prec, outer_rtol=1e-8, max_outer=40)
                row[name + ("_mixed" if prec else "")] = {
                    "status": int(st), "iterations": info["iterations"], "outer": info["outer"],
                    "ms": round(info["ms_total"], 1), "true_relres": info["true_relres"]}
            op.close()
        rows.append(row)
        print(json.dumps(row), flush=True)
    # the (1,1)-block scaling tau (tau = 1: the final proposition of Sec. 2.3; tau = 2: Prop. 2's
    # optimum for exact blocks) on the C1 and C2 shapes, smoothed W-cycle
    taus = []
    # ... and at every degree of the study on the metric recipe (32^3, two smoothed levels)
    vx, vy, vz, alpha, beta = workload(32)
    for k in (2, 3, 4, 5):
        for tau in (1.0, 2.0):
            op = hd.Operator(32, 32, 32, k, vx, vy, vz, alpha, beta, kind=hd.HD_GRAD_DIV, ess_mask=ESS, q=k + 2,
                             tau=tau, cycle=2, fp64_emulation=1, smooth_levels=2, stream=stream)
            b = torch.from_numpy(synth.uniform(op.n, seed=SEED + 7)).cuda()
            b[torch.from_numpy(op.hd_get_ess_dofs()).cuda()] = 0.0
            x = torch.zeros_like(b)
            st, info = op.hd_minres_solve(b, x, rtol=1e-8, maxit=args.solve_maxit, check_every=16,
                                          outer_rtol=1e-8, max_outer=40)
            taus.append({"shape": "tau_degree", "k": k, "tau": tau, "status": int(st),
                         "iterations": info["iterations"], "true_relres": info["true_relres"]})
            print(json.dumps(taus[-1]), flush=True)
            op.close()
    n1 = 4
    c1 = dict(nx=n1, k=2, q=3, kind=hd.HD_GRAD_DIV, ess=63, affine=True, rtol=1e-10,
              v=synth.lattice_vertices(n1, n1, n1), c0=np.ones(n1 ** 3), c1=np.ones(n1 ** 3))
    n2 = 32
    c2 = dict(nx=n2, k=3, q=5, kind=hd.HD_DARCY, ess=0, affine=False, rtol=1e-8,
              v=synth.lattice_vertices(n2, n2, n2, perturb=0.15, seed=SEED),
              c0=synth.lognormal(n2 ** 3, 2.0, seed=SEED + 1), c1=np.zeros(n2 ** 3))
    for name, c in (("C1", c1), ("C2", c2)):
        for tau in (1.0, 2.0):
            nx = c["nx"]
            op = hd.Operator(nx, nx, nx, c["k"], *c["v"], c["c0"], c["c1"], kind=c["kind"], ess_mask=c["ess"],
                             q=c["q"], affine=c["affine"], tau=tau, cycle=2, fp64_emulation=1, smooth_levels=2,
                             coarse_max=8 if nx < 8 else 0, stream=stream)
            b = torch.from_numpy(synth.uniform(op.n, seed=SEED + 7)).cuda()
            b[torch.from_numpy(op.hd_get_ess_dofs()).cuda()] = 0.0
            x = torch.zeros_like(b)
            st, info = op.hd_minres_solve(b, x, rtol=c["rtol"], maxit=args.solve_maxit, check_every=16,
                                          outer_rtol=c["rtol"], max_outer=40)
            taus.append({"shape": name, "tau": tau, "status": int(st), "iterations": info["iterations"],
                         "true_relres": info["true_relres"]})
            print(json.dumps(taus[-1]), flush=True)
            op.close()
    print(json.dumps({"study": "MINRES iterations vs mesh size and degree", "solver": "FP64 (double-float "
                      "element kernel), W-cycle, true relative residual 1e-8", "rows": rows, "tau": taus}),
          flush=True)


def run_winv_study(args):
    """W^-1 alternatives (Sec. 3.1 and its mass-inverse table): on perturbed meshes of about
    1.7 M L2 DOFs for k = 2..5, the setup of the W^-1 data and 100 applications of W^-1
    (hd_apply_C, FP64) by the stored explicit inverse (batched gemv), the stored Cholesky
    factors (two triangular solves), the fused local CG in the Gauss-Legendre nodal basis
    and the same CG in the histopolation basis; then the same four approaches for every
    degree of the paper's table, k = 2..9, through the degree-generic mass inverse."""
    import torch
    import paper_2304_12387_gb300 as hd
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    stream = torch.cuda.current_stream()
    rows = []
    for k, nx in ((2, 60), (3, 40), (4, 30), (5, 24)):
        vx, vy, vz, alpha, beta = workload(nx)
        row = {"k": k, "elements": nx ** 3, "l2_dofs": (nx * k) ** 3}
        ref = None
        for name, mode in (("inverse", hd.HD_WINV_DENSE), ("cholesky", hd.HD_WINV_CHOL), ("cg_gl", hd.HD_WINV_CG),
                           ("cg_hist", hd.HD_WINV_CG_HIST)):
            op = hd.Operator(nx, nx, nx, k, vx, vy, vz, alpha, beta, kind=hd.HD_GRAD_DIV, ess_mask=ESS, q=k + 2,
                             winv_mode=mode, stream=stream)
            st = op.hd_get_setup_times()
            q = torch.from_numpy(synth.uniform(op.n_l2, seed=SEED + 9)).cuda()
            y = torch.empty_like(q)
            for _ in range(3):
                op.hd_apply_C(q, y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(100):
                op.hd_apply_C(q, y)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            yh = y.cpu().numpy()
            if ref is None:
                ref = yh
            row[name] = {"setup_ms": round(st["winv"], 3), "solve_x100_ms": round(ms, 3),
                         "total_ms": round(st["winv"] + ms, 3), "gdof_s": round(op.n_l2 * 100 / ms / 1e6, 3),
                         "max_rel_diff_vs_inverse": float(np.abs(yh - ref).max() / np.abs(ref).max())}
            op.close()
        rows.append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps({"study": "W^-1 setup and 100 applications, FP64, perturbed mesh, q = k + 2",
                      "rows": rows}), flush=True)
    # every degree of the paper's table (p = k - 1 = 1..8) through the degree-generic mass
    # inverse (hd_massinv_*), about 1.7 M L2 DOFs each
    rows = []
    for k, nx in ((2, 60), (3, 40), (4, 30), (5, 24), (6, 20), (7, 17), (8, 15), (9, 13)):
        vx, vy, vz, alpha, _ = workload(nx)
        row = {"k": k, "p": k - 1, "elements": nx ** 3, "l2_dofs": (nx * k) ** 3}
        ref = None
        for name, mode, emul in (("inverse", hd.HD_WINV_DENSE, 0), ("cholesky", hd.HD_WINV_CHOL, 0),
                                 ("cg_gl", hd.HD_WINV_CG, 0), ("cg_hist", hd.HD_WINV_CG_HIST, 0),
                                 ("cg_gl_df", hd.HD_WINV_CG, 1)):
            mi = hd.MassInverse(nx, nx, nx, k, vx, vy, vz, alpha=alpha, method=mode, fp64_emulation=emul,
                                stream=stream)
            q = torch.from_numpy(synth.uniform(mi.n_l2, seed=SEED + 9)).cuda()
            y = torch.empty_like(q)
            for _ in range(3):
                mi.apply(q, y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(100):
                mi.apply(q, y)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            yh = y.cpu().numpy()
            if ref is None:
                ref = yh
            setup = mi.setup_ms()
            row[name] = {"setup_ms": round(setup, 3), "solve_x100_ms": round(ms, 3), "total_ms": round(setup + ms, 3),
                         "gdof_s": round(mi.n_l2 * 100 / ms / 1e6, 3), "cg_iterations": mi.iterations(),
                         "max_rel_diff_vs_inverse": float(np.abs(yh - ref).max() / np.abs(ref).max())}
            mi.close()
            del q, y
        rows.append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps({"study": "DG mass inverse of any degree (hd_massinv_*): setup and 100 applications, FP64 "
                               "(cg_gl_df: the CG stages in double-float), perturbed mesh, q = k + 2, alpha = 1",
                      "rows": rows}), flush=True)


def learned_study(args, stream):
    """The learned Schur preconditioner (P = V + network on the V/W-cycle V) on the Darcy
    recipe of its configuration: k = 3, perturbed mesh (+-15% h), eps = exp(2Z) per
    element, gamma = 0, natural BC. Trained on residual/correction pairs from the plain
    solver at 32^3 and then 64^3 elements, evaluated at 96^3 (95.8 M DOFs): time to a true
    relative residual of 1e-8 for FP64 MINRES with the V/W-cycle, mixed-precision MINRES
    with the V/W-cycle, and mixed-precision MINRES with the V/W-cycle plus the network
    (FP32 operator and cycle, FP16 network, FP64 residual correction), with iteration
    counts, the network's training losses and each solution's difference to the FP64
    one."""
    import torch
    import paper_2304_12387_gb300 as hd

    def darcy(n):
        vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=PERTURB, seed=SEED)
        return hd.Operator(n, n, n, 3, vx, vy, vz, synth.lognormal(n ** 3, SIGMA, seed=SEED + 1), np.zeros(n ** 3),
                           kind=hd.HD_DARCY, ess_mask=0, q=5, cycle=args.cycle, smooth_levels=args.smooth_levels,
                           fp64_emulation=1, stream=stream)

    def solve(op, b, precision, ref=None):
        x = torch.zeros_like(b)
        st, info = op.hd_minres_solve(b, x, rtol=1e-8 if precision == 0 else args.inner_rtol, maxit=args.solve_maxit,
                                      check_every=16, precision=precision, outer_rtol=1e-8, max_outer=40)
        r = {"status": int(st), "iterations": info["iterations"], "outer": info["outer"], "ms": info["ms_total"],
             "true_relres": info["true_relres"], "fallback": info["fallback"]}
        if ref is not None:
            r["rel_diff_vs_fp64_solution"] = float(torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref))
        return r, x

    out = {"workload": "Darcy k=3, q=5, +-15% h perturbed, eps=exp(2Z), gamma=0, natural BC; train 32^3 then 64^3 "
                       "elements, evaluate 96^3 (C5)",
           "preconditioner": "P = V + s C1^T C2^T C2 C1 s (V: the V/W-cycle; C1 3^3 conv 1->32, C2 3^3 conv 32->32, "
                             "FP16 weights and activations, FP32 accumulation)"}
    W = None
    for n, npairs, every, steps, lr in ((32, 8, 6, 100, 3e-3), (64, 6, 8, 50, 1e-3)):
        op = darcy(n)
        op.hd_learned_init()
        if W is not None:
            op.hd_learned_set_weights(*W)
        t = op.hd_learned_train(npairs=npairs, capture_every=every, steps=steps, lr=lr)
        out["train%d" % n] = {k: t[k] for k in ("pairs", "loss_initial", "loss_final", "ms_total")}
        W = op.hd_learned_get_weights()
        op.close()
    op = darcy(96)
    out["dofs"] = op.n
    op.hd_learned_init()
    op.hd_learned_set_weights(*W)
    b = torch.from_numpy(synth.uniform(op.n, seed=SEED + 9)).cuda()
    # the network alone (FP64 L2 vector in and out), per engine of its 32 -> 32 convolutions
    r = b[op.n_rt:].contiguous()
    zn = torch.empty_like(r)
    out["net_apply_ms"] = {}
    for name, engine in (("mma_sync", 1), ("tcgen05", 0)):
        op.hd_learned_conv_engine(engine)
        for _ in range(3):
            op.hd_learned_apply(r, zn)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(10):
            op.hd_learned_apply(r, zn)
        e1.record(stream)
        torch.cuda.synchronize()
        out["net_apply_ms"][name] = round(e0.elapsed_time(e1) / 10, 3)
    out["net_apply_ms"]["cells"] = int(op.n_l2)
    out["plain_fp64"], x64 = solve(op, b, 0)
    out["plain_mixed"], _ = solve(op, b, 1, x64)
    op.hd_set_schur_prec(1)
    out["learned_mixed"], _ = solve(op, b, 1, x64)
    op.hd_set_schur_prec(0)
    op.close()
    # the element-aligned hierarchy (odd k: no aggregate straddles an element boundary), one
    # smoothed level: the plain cycle at its best on this degree
    vx, vy, vz = synth.lattice_vertices(96, 96, 96, perturb=PERTURB, seed=SEED)
    op = hd.Operator(96, 96, 96, 3, vx, vy, vz, synth.lognormal(96 ** 3, SIGMA, seed=SEED + 1), np.zeros(96 ** 3),
                     kind=hd.HD_DARCY, ess_mask=0, q=5, cycle=args.cycle, smooth_levels=1, aggregation=1,
                     fp64_emulation=1, stream=stream)
    out["aligned_fp64"], _ = solve(op, b, 0, x64)
    out["aligned_mixed"], _ = solve(op, b, 1, x64)
    op.close()
    lm, pf, pm = out["learned_mixed"], out["plain_fp64"], out["plain_mixed"]
    out["learned_mixed_vs_plain_fp64"] = {"time_ratio": lm["ms"] / pf["ms"], "speedup": pf["ms"] / lm["ms"]}
    out["learned_mixed_vs_plain_mixed"] = {"iteration_ratio": lm["iterations"] / max(1, pm["iterations"]),
                                           "time_ratio": lm["ms"] / pm["ms"]}
    return out


def run_net_apply(args):
    """The learned network alone on the Darcy recipe of the learned study (k = 3,
    +-15% h, eps = exp(2Z)) at n^3 elements, untrained initial weights: milliseconds per
    application of P_L (FP64 L2 vector in and out) with the 32 -> 32 convolutions on
    the tcgen05 tensor cores and with mma.sync, and the rate of those two convolutions
    (2 x 2 x 32 x 32 x 27 flops per cell per application)."""
    import torch
    import paper_2304_12387_gb300 as hd
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    stream = torch.cuda.current_stream()
    n = args.net_apply
    vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=PERTURB, seed=SEED)
    op = hd.Operator(n, n, n, 3, vx, vy, vz, synth.lognormal(n ** 3, SIGMA, seed=SEED + 1), np.zeros(n ** 3),
                     kind=hd.HD_DARCY, ess_mask=0, q=5, cycle=2, smooth_levels=2, fp64_emulation=1, stream=stream)
    op.hd_learned_init()
    r = torch.from_numpy(synth.uniform(op.n_l2, seed=SEED + 3)).cuda()
    z = torch.empty_like(r)
    out = {"study": "learned network apply", "elements": n ** 3, "cells": op.n_l2}
    for name, engine in (("mma_sync", 1), ("tcgen05", 0)):
        op.hd_learned_conv_engine(engine)
        for _ in range(3):
            op.hd_learned_apply(r, z)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            op.hd_learned_apply(r, z)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out[name] = {"ms_per_apply": round(ms, 4)}
    out["conv_flops_per_apply"] = 2 * 2 * 32 * 32 * 27 * op.n_l2
    out["tc_status"] = int(op.hd_tc_status())
    op.close()
    print(json.dumps(out), flush=True)


def run_raddiff(args):
    """Grey nonlinear radiation diffusion (Sec. 4.3) on the perturbed mesh of the metric
    recipe at n^3 elements, k = 4: a hot spot T = 1 + exp(-30 |x - x_c|^2) in cold radiation
    (E = a), opacity sigma = exp(0.5 Z) per element, rho = Cv = a = c = 1, reflecting walls,
    dt = h (the paper's dt = h / tau for a solution decaying at rate tau = 1), no sources.
    Time, phase shares and iteration counts of --rad-steps SDIRK3 steps, with the stage
    tolerances of the paper (outer 1e-12, Newton 1e-8, linear 1e-8)."""
    import torch
    import paper_2304_12387_gb300 as hd
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    stream = torch.cuda.current_stream()
    n = args.raddiff
    vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=PERTURB, seed=SEED)
    E = n ** 3
    sigma = synth.lognormal(E, 0.5, seed=SEED + 7)
    t0 = time.time()
    rd = hd.RadDiff(n, n, n, K, vx, vy, vz, sigma, 1.0 / n, rho=1.0, cv=1.0, a=1.0, c=1.0, cycle=args.cycle,
                    smooth_levels=args.smooth_levels, fp64_emulation=args.fp64_emulation,
                    linear_rtol=args.rad_linear_rtol, linear_precision=args.rad_linear_precision, stream=stream)
    setup_s = time.time() - t0
    nl = rd.n_l2
    X = rd.points()
    T0 = 1.0 + np.exp(-30.0 * np.sum((X - 0.5) ** 2, axis=-1))
    del X
    e, Eh, tmp, Ev = (torch.empty(nl, dtype=torch.float64, device="cuda") for _ in range(4))
    rd.load(torch.from_numpy(T0).cuda(), tmp)
    rd.winv(tmp, e)
    rd.load(torch.ones(E, rd.q ** 3, dtype=torch.float64, device="cuda"), Eh)
    F = torch.zeros(rd.n_rt, dtype=torch.float64, device="cuda")

    def energy():
        rd.winv(Eh, Ev)
        return e.sum().item() + Ev.sum().item()

    W0 = energy()
    tot = {"stages": 0, "outer": 0, "outer_max": 0, "newton_max": 0, "linear_solves": 0, "linear_iterations": 0,
           "relres": 0.0, "ms_newton": 0.0, "ms_linear": 0.0, "ms_residual": 0.0}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.rad_steps):
        info = rd.step(e, Eh, F)
        for key in ("stages", "outer", "linear_solves", "linear_iterations", "ms_newton", "ms_linear",
                    "ms_residual"):
            tot[key] += info[key]
        for key in ("outer_max", "newton_max", "relres"):
            tot[key] = max(tot[key], info[key])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    phases = tot["ms_newton"] + tot["ms_linear"] + tot["ms_residual"]
    out = {"study": "radiation diffusion (Sec. 4.3)", "elements": E, "k": K, "n_rt": rd.n_rt, "n_l2": nl,
           "linear_rtol": args.rad_linear_rtol, "linear_precision": args.rad_linear_precision,
           "dofs": rd.n_rt + nl, "dt": 1.0 / n, "steps": args.rad_steps, "setup_s": round(setup_s, 3),
           "ms_total": round(ms, 1), "ms_per_stage": round(ms / max(tot["stages"], 1), 1),
           "share": {"nonlinear_residual": round(tot["ms_residual"] / phases, 4),
                     "inner_newton": round(tot["ms_newton"] / phases, 4),
                     "linear_solver": round(tot["ms_linear"] / phases, 4)},
           "minres_iterations_per_solve": round(tot["linear_iterations"] / max(tot["linear_solves"], 1), 1),
           "outer_per_stage": round(tot["outer"] / max(tot["stages"], 1), 2),
           "energy_drift": abs(energy() - W0) / abs(W0), **tot,
           "paper_context": {"hardware": "16 V100", "elements": 884736, "share": {
               "nonlinear_residual": 0.0445, "inner_newton": 0.0387, "linear_solver": 0.9168},
               "minres_iterations_per_solve": 84, "outer_per_stage": 2}}
    rd.close()
    out["value"] = out["dofs"] * args.rad_steps / (ms * 1e-3)
    out["unit"] = "DOF-steps/s"
    if not args.no_cpu:
        out["cpu_baseline"] = rad_cpu_baseline(1.0 / n)
    print(json.dumps(out), flush=True)


def _rad_oracle_worker(arg):
    """The oracle's SDIRK3 step on an n^3-element sample of the radiation-diffusion recipe
    with the time step dt of the measured workload (one process, one thread): (DOFs,
    seconds for the step, passes per stage)."""
    from oracle.raddiff import RadDiff
    n, dt = arg
    vx, vy, vz = synth.lattice_vertices(n, n, n, perturb=PERTURB, seed=SEED)
    sigma = synth.lognormal(n ** 3, 0.5, seed=SEED + 7)
    rd = RadDiff(n, n, n, K, vx, vy, vz, sigma, dt, q=Q)
    X = rd.points()
    e = rd.project(1.0 + np.exp(-30.0 * np.sum((X - 0.5) ** 2, axis=-1)))
    Eh = rd.load(np.ones(X.shape[:2]))
    F = np.zeros(rd.n_rt)
    t0 = time.perf_counter()
    _, _, _, infos = rd.step(e, Eh, F)
    return rd.n_rt + rd.n_l2, time.perf_counter() - t0, sum(i["outer"] for i in infos) / 3.0


def rad_cpu_baseline(dt, n=4):
    """The oracle's radiation-diffusion step timed on one host core (a spawned process with
    one BLAS thread), on an n^3-element sample of the same recipe and time step."""
    import multiprocessing as mp
    saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for v in saved:
        os.environ[v] = "1"
    try:
        with mp.get_context("spawn").Pool(1) as pool:
            dofs, sec, passes = pool.apply(_rad_oracle_worker, ((n, dt),))
    finally:
        for v, old in saved.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old
    return {"value": dofs / sec, "unit": "DOF-steps/s", "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": "%d^3 elements of the same recipe and dt (%d DOFs): one SDIRK3 step, dense Newton systems "
                      "and a sparse LU of the Darcy system, %.2f s, %.1f passes per stage" % (n, dofs, sec, passes)}


def run_learned(args):
    """The learned-preconditioner study alone (one JSON line)."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    print(json.dumps({"metric": "learned Schur preconditioner: MINRES time to a true 1e-8",
                      **learned_study(args, torch.cuda.current_stream())}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--inner-rtol", type=float, default=1e-4, help="inner MINRES tolerance of the mixed solve")
    ap.add_argument("--solve-maxit", type=int, default=20000, help="iteration cap of the MINRES solves")
    ap.add_argument("--cycle", type=int, default=2, choices=[1, 2], help="1: V-cycle, 2: W-cycle on S~")
    ap.add_argument("--smooth-levels", type=int, default=2, choices=[0, 1, 2],
                    help="smoothed-aggregation prolongators on the first 1 or 2 levels of the S~ hierarchy "
                         "(0: plain aggregation)")
    ap.add_argument("--w-levels", type=int, default=0, help="W repetition on the first levels only (0: all)")
    ap.add_argument("--learned", action="store_true", help="run the learned-preconditioner study alone")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner study")
    ap.add_argument("--gmres-restart", type=int, default=32, help="GMRES restart length (block-triangular solve)")
    ap.add_argument("--solvers", default="minres,gmres",
                    help="comma-separated solves of the timed line: minres (FP64 and mixed), gmres (FP64 and mixed)")
    ap.add_argument("--gmres-inner-rtol", type=float, default=1e-3,
                    help="per-cycle reduction of the mixed-precision GMRES before its FP64 residual")
    ap.add_argument("--winv-study", action="store_true",
                    help="W^-1 by explicit inverse, Cholesky and local CG (GL and histopolation bases): setup "
                         "and 100 applies")
    ap.add_argument("--iterations", action="store_true",
                    help="run the iteration-count study (mesh sizes and degrees) instead")
    ap.add_argument("--fp64-emulation", type=int, default=1, choices=[0, 1, 2],
                    help="1: element kernel in double-float (FP32 pairs, FP64 parity); 2: and the Schur cycle of "
                         "the FP64 preconditioner; 0: native FP64")
    ap.add_argument("--no-native", action="store_true", help="skip the native-FP64 comparison apply")
    ap.add_argument("--no-affine", action="store_true", help="skip the apply on the unperturbed (affine) mesh")
    ap.add_argument("--n", type=int, default=NX, help="elements per direction (64 = the metric workload)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--raddiff", type=int, default=0,
                    help="run the radiation-diffusion study alone at this many elements per direction (k = 4)")
    ap.add_argument("--rad-steps", type=int, default=1, help="SDIRK3 steps of the radiation-diffusion study")
    ap.add_argument("--rad-linear-precision", type=int, default=0, choices=[0, 1],
                    help="Darcy solves of the radiation-diffusion study: 0 FP64 MINRES, 1 mixed precision")
    ap.add_argument("--rad-linear-rtol", type=float, default=1e-8,
                    help="MINRES tolerance of each Darcy solve in the radiation-diffusion study (paper: 1e-8)")
    ap.add_argument("--net-apply", type=int, default=0,
                    help="time the learned network alone at this many elements per direction (k = 3)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", 1))
    rank = int(os.environ.get("RANK", 0))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl" if args.impl == "ours" else "gloo")
        dist = tdist
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.learned:
        run_learned(args)
    elif args.iterations:
        run_iterations(args)
    elif args.net_apply:
        run_net_apply(args)
    elif args.raddiff:
        run_raddiff(args)
    elif args.winv_study:
        run_winv_study(args)
    else:
        run_ours(args, rank, world, dist)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
