"""Benchmark of the HDArray hot path on GB300.

Headline workload (one "step"): 2-D 5-point Jacobi on an 8192 x 8192 binary32 grid split 4 x 4
(BLOCK) over 16 logical devices, the paper's data/work partition pair (whole grid / interior),
100 Jacobi iterations (exchange of the +-1 halo fused into the stencil launch, all 16 devices in
one launch per iteration, replayed from a CUDA graph of two iterations), then the binary64
residual sum((A - B)^2) via HDArrayReduce.  Inputs (2 x 268 MB) exceed the 129 MB L2, so no flush
is needed between steps.

The same JSON line carries one sub-record per other workload (key "workloads"): the 256^2 binary64
Jacobi (ROW 4, 10 iterations + residual), the 512^3 3-D 7-point stencil over 37 uneven boxes
(50 iterations), the triangular GEMM tril(A) 8192^2 x B 8192x4096 over 8 row partitions (binary64
DFMA, bf16x3 and bf16x6 on the tensor cores, the B all-gather alone), and the batch of 512 Jacobi
instances (200 iterations, one launch per iteration).  Each has its CUDA-event time, its roofline
and a parity check against an independent numpy evaluation run in the same process.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

Prints one JSON line.  With N > 1 (torchrun) every rank runs an independent replica (the
single-GPU partitions do not span GPUs); the value is the sum over ranks of the work divided by
the slowest rank's time.
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

METRIC = "stencil Gcell-updates/s + exchange GB/s vs HBM peak; batched/mixed vs plain form"
UNIT = "Gcell-updates/s"
N, P, ITERS = 8192, 16, 100
CELLS = (N - 2) * (N - 2)
WORKLOAD = ("2-D 5-point Jacobi 8192x8192 FP32, 4x4 BLOCK = 16 logical devices, +-1 halo, "
            "100 iterations per step (exchange fused, one launch per iteration, CUDA graph) "
            "+ FP64 residual via HDArrayReduce")
PROFILES = os.path.join(ROOT, "profiles")
CSRC = os.path.join(ROOT, "paper_1809_05657_gb300", "csrc")


# ---------------------------------------------------------------------------------------------
# peaks, profiles, clocks
# ---------------------------------------------------------------------------------------------

def peaks():
    """Measured denominators: HBM copy GB/s and cuBLAS bf16 TFLOP/s (burst, sustained)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm": float(d["hbm_gbs"]), "bf16": float(d["bf16_tflops"]),
                "bf16_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    except Exception:
        return {"hbm": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


def code_hash(sources):
    """First 16 hex digits of the SHA-256 of the kernel sources' code: each file with its `//`
    comments, trailing blanks and empty lines removed, so that a comment edit does not make a
    profile stale while any change to the code does."""
    h = hashlib.sha256()
    for src in sources:
        for line in open(os.path.join(CSRC, src), encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode("utf-8") + b"\n")
    return h.hexdigest()[:16]


def profiled(name, key, sources):
    """A figure from the committed ncu summary profiles/<name>: the value of `- key: value` in its
    "Values read by bench.py" list, or None when the kernel sources' code changed since the capture
    (the summary records code_hash(sources)) or the key is absent."""
    try:
        txt = open(os.path.join(PROFILES, name)).read()
        vals = {}
        for line in txt.splitlines():
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip()
        if vals.get("kernel_code_sha256_16") != code_hash(sources):
            return None
        return float(vals[key])
    except Exception:
        return None


KERNEL_NAMES_2D = {0: "k_jacobi2d<f32,6> (register ring)", 1: "k_jacobi2d_async<f32,8> (cp.async ring)",
                   2: "k_jacobi2d_flat<f32>", 3: "k_jacobi2d_cta<f32,8> (packed row streams)",
                   5: "k_jacobi2d_tma<f32,4,4> (rows staged by bulk tensor copies)"}


def jacobi_variant(tuned, dtype="f32"):
    """The 2-D kernel variant the headline workload ran: the tuner's choice for its storage type,
    else the environment's or the library default."""
    for t in tuned or []:
        if t.get("kernel") == "jacobi2d" and t.get("dtype") == dtype:
            return int(t["variant"])
    try:
        v = int(os.environ.get("HDARRAY_JACOBI_VARIANT", "1"))
        return v if v in KERNEL_NAMES_2D else 1
    except ValueError:
        return 1


def stencil3d_variant():
    """The 3-D kernel variant this run used: the tuner's choice (from the run's tuning file), else
    the environment's or the library default (1)."""
    for t in tune_report(os.environ.get("HDARRAY_TUNE_CACHE")) or []:
        if t.get("kernel") == "stencil3d" and t.get("dtype") == "f32":
            return int(t["variant3"])
    try:
        return int(os.environ.get("HDARRAY_STENCIL3D_VARIANT", "1"))
    except ValueError:
        return 1


def conv_variant():
    """The convolution kernel this run used: variant 5 (rows staged by TMA) or 3 (packed streams)."""
    for t in tune_report(os.environ.get("HDARRAY_TUNE_CACHE")) or []:
        if t.get("kernel") == "conv2d" and t.get("dtype") == "f32":
            return int(t["variant"])
    return 5 if os.environ.get("HDARRAY_JACOBI_VARIANT") == "5" else 3


class ClockSampler:
    """nvidia-smi clock and throttle samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# independent numpy evaluations for the in-run parity checks (not the oracle)
# ---------------------------------------------------------------------------------------------

def stencil_steps(w, iters, ft):
    """`iters` steps of the printed stencil on the array w in arithmetic type ft, updating every
    cell that is not on w's outer ring: 2-D ((W + E) + N) + S, times 1/4 (Sec. 5); 3-D the six
    face neighbours x-, x+, y-, y+, z-, z+ summed in that order, then one division by 6."""
    import numpy as np
    w = np.array(w, dtype=ft)
    for _ in range(iters):
        new = w.copy()
        if w.ndim == 2:
            s = w[1:-1, :-2] + w[1:-1, 2:]
            s = s + w[:-2, 1:-1]
            s = s + w[2:, 1:-1]
            new[1:-1, 1:-1] = s * ft(0.25)
        else:
            s = w[1:-1, 1:-1, :-2] + w[1:-1, 1:-1, 2:]
            s = s + w[1:-1, :-2, 1:-1]
            s = s + w[1:-1, 2:, 1:-1]
            s = s + w[:-2, 1:-1, 1:-1]
            s = s + w[2:, 1:-1, 1:-1]
            new[1:-1, 1:-1, 1:-1] = s / ft(6.0)
        w = new
    return w


def light_cone(x0, pt, iters, ft):
    """Value at pt after `iters` stencil steps of the whole array x0 (its outer ring fixed),
    evaluated on the window of cells within `iters` + 1 of pt: the window's edge cells are never
    updated, and what that gets wrong moves inward one cell per step, never reaching pt."""
    lo = [max(0, p - iters - 1) for p in pt]
    hi = [min(n, p + iters + 2) for p, n in zip(pt, x0.shape)]
    w = stencil_steps(x0[tuple(slice(a, b) for a, b in zip(lo, hi))], iters, ft)
    return w[tuple(p - a for p, a in zip(pt, lo))]


def cone_check(x0, got, pts, iters, ft32):
    """Bit-exact comparison of sampled cells with the same-precision evaluation, and the relative
    error (max |x - x*| / max |x*|) against binary64."""
    import numpy as np
    exact, err, mag = 0, 0.0, 0.0
    for pt in pts:
        g = got[tuple(pt)]
        exact += int(np.array(light_cone(x0, pt, iters, ft32), ft32).tobytes() == np.array(g, ft32).tobytes())
        r64 = float(light_cone(x0, pt, iters, np.float64))
        err = max(err, abs(float(g) - r64))
        mag = max(mag, abs(r64))
    return {"samples": len(pts), "bit_exact_same_precision": exact,
            "err_vs_binary64": err / mag if mag else err,
            "reference": "numpy light-cone evaluation in the same precision and in binary64"}


# ---------------------------------------------------------------------------------------------
# the headline workload
# ---------------------------------------------------------------------------------------------

def setup_jacobi(H, dtype):
    B = H.HDArrayCreate("B", dtype, None, N, N)
    A = H.HDArrayCreate("A", dtype, None, N, N)
    R = H.HDArrayCreate("R", "double", None, N, N)
    D = H.HDArrayPartition(H.BLOCK, (N, N), (0, 0), (N, N), P)
    W = H.HDArrayPartition(H.BLOCK, (N, N), (1, 1), (N - 1, N - 1), P)
    return B, A, R, D, W


def tune_setup(args):
    """Autotuning of the stencil tile shapes (the library times candidates on first use); the
    choices are appended to a per-run file whose lines are reported in the JSON."""
    if args.no_autotune:
        return None
    path = os.path.join("/tmp", "hdarray_tune_%d.txt" % os.getpid())
    if os.path.exists(path):
        os.remove(path)
    os.environ["HDARRAY_AUTOTUNE"] = "1"
    os.environ["HDARRAY_TUNE_CACHE"] = path
    return path


def tune_report(path):
    if not path or not os.path.exists(path):
        return None
    out = []
    for line in open(path):
        w = line.split()
        if len(w) == 10:
            key = w[0].split(":")
            out.append({"kernel": key[0], "dtype": {"0": "f64", "1": "f32", "2": "bf16"}.get(key[1] if len(key) > 1 else "", "?"),
                        "variant": int(w[1]), "rows": int(w[2]), "warps": int(w[3]),
                        "tile_z": int(w[4]), "fused_exchange": int(w[5]), "variant3": int(w[6]),
                        "band3": int(w[7]), "cta3": int(w[8]), "band2": int(w[9])})
    return out


def max_over_ranks(ms, world, device):
    """The slowest rank's time: every replica's timed region ends before the job's does."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, world, ms):
    """Whole-job rate of `world` independent replicas that each processed units_per_rank units
    in at most ms milliseconds (weak scaling: the per-GPU work is fixed)."""
    return world * units_per_rank / (ms * 1e-3)


def gpu_arm(args, rank, world):
    import numpy as np
    import torch
    from __graft_entry__ import build_library
    from paper_1809_05657_gb300 import hdarray as H
    import synthetic

    build_library()
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    H.HDArrayInit(ndev=P)
    H.HDArraySetStream(stream.cuda_stream)
    storage = args.storage
    esize = 4 if storage == "float" else 2
    x = synthetic.jacobi_field((N, N), stream=1, dtype=storage)
    xh = torch.from_numpy(x if storage == "float" else x.view(np.int16)).pin_memory()
    B, A, R, D, W = setup_jacobi(H, storage)
    H.HDArrayWrite(B, xh, D)

    def warm_iters(b, a):
        H.HDArrayApplyKernel("jacobi2d", W, b, a)
        H.HDArrayApplyKernel("jacobi2d", W, a, b)

    for _ in range(2):
        warm_iters(B, A)
    H.HDArrayGraphBegin()
    warm_iters(B, A)
    gid = H.HDArrayGraphEnd()

    def residual():
        H.HDArrayApplyKernel("sqdiff", W, B, A, R)
        return H.HDArrayReduce(R, H.SUM, W)

    # exchange volume of one iteration (the fused kernel's halo traffic)
    H.HDArrayApplyKernel("jacobi2d", W, B, A)
    xbytes = sum(int(np.prod(np.subtract(hi, lo))) for _, _, lo, hi in H.HDArrayGetPlan(B)) * esize
    H.HDArrayApplyKernel("jacobi2d", W, A, B)
    torch.cuda.synchronize()

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        H.HDArrayGraphLaunch(gid, ITERS // 2)
        if ev is not None:
            ev[1].record(stream)
        return residual()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    c0 = H.HDArrayGetCounters()
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = None
    with ClockSampler(dev) as clk:
        torch.cuda.synchronize()
        t0.record(stream)
        for k in range(args.steps):
            res = step(kev[k])
        t1.record(stream)
        torch.cuda.synchronize()
    c1 = H.HDArrayGetCounters()
    ms = max_over_ranks(t0.elapsed_time(t1), world, "cuda")
    kernel_ms = sum(a.elapsed_time(b) for a, b in kev)
    launches = c1["launches"] - c0["launches"]
    per_launch_ms = kernel_ms / (args.steps * ITERS)
    algo_bytes = CELLS * 2 * esize + 2 * xbytes
    pk = peaks()
    achieved = algo_bytes / (per_launch_ms * 1e-3) / 1e9
    value = replica_rate(CELLS * ITERS * args.steps, world, ms) / 1e9
    residual_us = (t0.elapsed_time(t1) - kernel_ms) / args.steps * 1e3

    e2e, parity = None, None
    if rank == 0 and not args.quick and storage == "float":
        e2e = e2e_run(H, torch, stream, B, A, R, D, W, xh, gid, args)
        # a fresh step from the input: the field after exactly 100 iterations
        H.HDArrayWrite(B, xh, D)
        for _ in range(2):
            H.HDArrayApplyKernel("jacobi2d", W, B, A)
            H.HDArrayApplyKernel("jacobi2d", W, A, B)
        H.HDArrayGraphLaunch(gid, (ITERS - 4) // 2)
        got = np.zeros((N, N), np.float32)
        H.HDArrayRead(B, got, D)
        parity = cone_check(x, got, sample_points_2d(N), ITERS, np.float32)
    H.HDArrayExit()
    extra = {}
    if rank == 0 and not args.quick and storage == "float":
        extra = extra_forms(H, torch, stream, args)
    return dict(ms=ms, value=value, launches=launches, per_launch_ms=per_launch_ms,
                algo_bytes=algo_bytes, xbytes=xbytes, achieved=achieved, peaks=pk,
                clocks=clk.summary(), residual=res, extra=extra, e2e=e2e, parity=parity,
                residual_us=residual_us)


def sample_points_2d(n):
    """Cells for the light-cone checks: next to the 4 x 4 block boundaries, the corners of the
    interior and a few seeded interior cells."""
    import synthetic
    b = [n * k // 4 for k in range(1, 4)]
    pts = [(b[0] - 1, b[0]), (b[1], b[1] - 1), (b[2], b[2]), (1, 1), (n - 2, n - 2), (1, n - 2),
           (b[1] - 1, 1), (n - 2, b[0])]
    u = synthetic.uniform(8, stream=901)
    pts += [(1 + int(u[i] * (n - 2)), 1 + int(u[i + 1] * (n - 2))) for i in range(0, 8, 2)]
    return pts


def e2e_run(H, torch, stream, B, A, R, D, W, xh, gid, args):
    """The step through the C ABI with host buffers, steps in a row as a time-stepping program runs
    them: HDArrayWrite of each step's input from pinned host memory, the 100 iterations, the
    residual back to the host (HDArrayReduce).  The inputs alternate between two arrays (B and a
    second one), so the Write of step k+1's input -- queued right after step k's iterations, on the
    library's copy stream -- overlaps step k's compute; the library orders it after the second
    array's last use and every later use after it.  Timed on the host around whole steps (each
    step's Reduce synchronises); the timed region holds every step's input copy, the first one
    included (nothing to overlap it with)."""
    B2 = H.HDArrayCreate("B2", "float", None, N, N)
    H.HDArrayWrite(B2, xh, D)
    for _ in range(2):
        H.HDArrayApplyKernel("jacobi2d", W, B2, A)
        H.HDArrayApplyKernel("jacobi2d", W, A, B2)
    H.HDArrayGraphBegin()
    H.HDArrayApplyKernel("jacobi2d", W, B2, A)
    H.HDArrayApplyKernel("jacobi2d", W, A, B2)
    gid2 = H.HDArrayGraphEnd()
    inputs, graphs = [B, B2], [gid, gid2]

    def run(steps):
        res = None
        H.HDArrayWrite(inputs[0], xh, D)                 # host -> device, 268 MB
        for k in range(steps):
            X, g = inputs[k % 2], graphs[k % 2]
            for _ in range(2):                            # back into the graph's periodic state
                H.HDArrayApplyKernel("jacobi2d", W, X, A)
                H.HDArrayApplyKernel("jacobi2d", W, A, X)
            H.HDArrayGraphLaunch(g, (ITERS - 4) // 2)
            if k + 1 < steps:                             # the next step's input, during this one
                H.HDArrayWrite(inputs[(k + 1) % 2], xh, D)
            H.HDArrayApplyKernel("sqdiff", W, X, A, R)
            res = H.HDArrayReduce(R, H.SUM, W)            # device -> host, 8 bytes
        return res
    run(max(2, args.warmup))
    torch.cuda.synchronize()
    steps = max(2, args.steps // 2)
    t0 = time.perf_counter()
    res = run(steps)
    ms = (time.perf_counter() - t0) * 1e3 / steps
    H.HDArrayFree(B2)
    return {"value": CELLS * ITERS / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "h2d_bytes_per_step": N * N * 4, "d2h_bytes_per_step": 8, "residual": res,
            "path": "HDArrayWrite(input, pinned host array, data partition) -> 100 iterations -> "
                    "HDArrayApplyKernel(sqdiff) -> HDArrayReduce (host double); inputs alternate between "
                    "two arrays so the next step's Write (library copy stream) overlaps this step's "
                    "compute; host wall clock"}


def extra_forms(H, torch, stream, args):
    """The comparison forms on the same GPU: BF16 storage (fused, graph) and the plain
    per-partition binary64 form of the paper's program (two kernels, one copy launch per
    section, one launch per device, no graph)."""
    import numpy as np
    import synthetic
    out = {}
    pk = peaks()
    H.HDArrayInit(ndev=P)
    H.HDArraySetStream(stream.cuda_stream)
    xb = synthetic.jacobi_field((N, N), stream=1, dtype="bf16")
    B, A, R, D, W = setup_jacobi(H, "bf16")
    H.HDArrayWrite(B, torch.from_numpy(xb.view(np.int16)).pin_memory(), D)
    for _ in range(2):
        H.HDArrayApplyKernel("jacobi2d", W, B, A)
        H.HDArrayApplyKernel("jacobi2d", W, A, B)
    H.HDArrayGraphBegin()
    H.HDArrayApplyKernel("jacobi2d", W, B, A)
    H.HDArrayApplyKernel("jacobi2d", W, A, B)
    gid = H.HDArrayGraphEnd()
    H.HDArrayGraphLaunch(gid, 10)
    ms = _events(torch, stream, lambda: H.HDArrayGraphLaunch(gid, 50), 1) / 100
    out["bf16_fused"] = {"gcells_per_s": CELLS / (ms * 1e-3) / 1e9, "us_per_iter": ms * 1e3,
                         "hbm_frac": CELLS * 4 / (ms * 1e-3) / 1e9 / pk["hbm"]}
    H.HDArrayExit()
    # plain binary64 form
    H.HDArrayInit(ndev=P)
    H.HDArraySetStream(stream.cuda_stream)
    H.HDArraySetMode(H.HDARRAY_MODE_PLAIN)
    x64 = synthetic.jacobi_field((N, N), stream=1, dtype="double")
    B, A, R, D, W = setup_jacobi(H, "double")
    H.HDArrayWrite(B, torch.from_numpy(x64).pin_memory(), D)
    for _ in range(2):
        H.HDArrayApplyKernel("jacobi2d", W, B, A)
        H.HDArrayApplyKernel("copy", W, A, B)
    torch.cuda.synchronize()
    it = 10
    c0 = H.HDArrayGetCounters()

    def plain():
        for _ in range(it):
            H.HDArrayApplyKernel("jacobi2d", W, B, A)
            H.HDArrayApplyKernel("copy", W, A, B)
    ms = _events(torch, stream, plain, 1) / it
    c1 = H.HDArrayGetCounters()
    # traffic of one plain iteration: the step (read B, write A) and the copy back (read A,
    # write B), 8 bytes each per cell
    gbs = CELLS * 32 / (ms * 1e-3) / 1e9
    out["plain_fp64"] = {"gcells_per_s": CELLS / (ms * 1e-3) / 1e9, "us_per_iter": ms * 1e3,
                         "launches_per_iter": (c1["launches"] - c0["launches"]) / it,
                         "hbm_frac_of_its_traffic": gbs / pk["hbm"],
                         "fp64_tflops": 5 * CELLS / (ms * 1e-3) / 1e12,
                         "note": "5 binary64 flops per cell update; traffic 32 B per cell (step + copy)"}
    H.HDArrayExit()
    return out


# ---------------------------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------------------------

SAMPLE_N = 2048


def _oracle_program(n, threads):
    """The Jacobi program of the headline workload on an n x n binary32 grid in the oracle:
    16-device BLOCK data/work partitions, the input written.  Returns (oracle, B, A, W, work mask,
    threads used)."""
    import numpy as np
    import oracle
    import synthetic
    used = oracle.set_threads(threads)
    o = oracle.Oracle(P)
    x = synthetic.jacobi_field((n, n), stream=1, dtype="float")
    B = o.create("B", "float", (n, n))
    A = o.create("A", "float", (n, n))
    D = o.partition(oracle.BLOCK, (n, n), (0, 0), (n, n))
    W = o.partition(oracle.BLOCK, (n, n), (1, 1), (n - 1, n - 1))
    o.write(B, x, D)
    work = np.zeros(n * n, np.uint8)
    for box in o.parts[W]:
        if box is not None:
            B.mask_box(box[0], box[1], work)
    return o, B, A, W, work, used


def _value_loops(n, iters, threads):
    """The oracle's Jacobi value loops (the compute of each apply) alone, ping-pong, `iters`
    iterations on the n x n grid.  Returns (seconds, cell updates, threads used)."""
    import ctypes
    import oracle
    o, B, A, W, work, used = _oracle_program(n, threads)
    L = oracle.lib()
    wp = work.ctypes.data_as(ctypes.c_void_p)
    b, a = B.G, A.G
    t = time.perf_counter()
    for _ in range(iters):
        L.orc_jacobi2d(1, n, n, b.ctypes.data_as(ctypes.c_void_p), a.ctypes.data_as(ctypes.c_void_p), wp)
        a, b = b, a
    sec = time.perf_counter() - t
    oracle.set_threads(1)
    return sec, (n - 2) * (n - 2) * iters, used


def _set_enumeration(n, iters):
    """The oracle's per-element def/use bookkeeping alone (messages of Eq. 1-2, GDEF update of
    Eq. 3-4, no values), `iters` ping-pong iterations on the n x n grid.  Returns seconds."""
    o, B, A, W, work, used = _oracle_program(n, 1)
    t = time.perf_counter()
    for _ in range(iters):
        o.apply("jacobi2d", W, [B, A], compute=False)
        A, B = B, A
    return time.perf_counter() - t


def cpu_baseline():
    """The oracle on the host cores: its Jacobi value loops on the full 8192 x 8192 grid on all
    cores (OpenMP) and on one core, and its per-element set enumeration timed separately."""
    ncores = os.cpu_count() or 1
    s_all, c_all, used = _value_loops(N, 12, ncores)
    s_one, c_one, _ = _value_loops(N, 3, 1)
    s_set = _set_enumeration(SAMPLE_N, 2)
    return {"value": c_all / s_all / 1e9, "unit": UNIT, "cores": used, "kind": "oracle", "nproc": ncores,
            "sample": "%dx%d FP32, the oracle's Jacobi value loops over the 16 devices' work regions, "
                      "12 iterations on %d threads (%.1f s)" % (N, N, used, s_all),
            "single_thread": {"value": c_one / s_one / 1e9, "unit": UNIT, "cores": 1,
                              "sample": "the same loops, 3 iterations on one thread (%.1f s)" % s_one},
            "set_enumeration": {"seconds_per_iteration": s_set / 2, "cells_per_s": (SAMPLE_N - 2) ** 2 * 2 / s_set,
                                "sample": "%dx%d, 16 devices, per-element messages and GDEF update "
                                          "(Eq. 1-4), 2 iterations, one thread" % (SAMPLE_N, SAMPLE_N)}}


def oracle_sample(iters, threads):
    """The whole oracle program on a bounded sample of the headline workload: a 2048 x 2048
    binary32 grid with the same 16-device BLOCK data/work partitions, `iters` ping-pong Jacobi
    iterations with per-element message generation and the value loops on `threads` threads.
    Returns (seconds, cell updates, threads used)."""
    o, B, A, W, work, used = _oracle_program(SAMPLE_N, threads)
    t = time.perf_counter()
    for _ in range(iters):
        o.apply("jacobi2d", W, [B, A])
        A, B = B, A
    sec = time.perf_counter() - t
    import oracle
    oracle.set_threads(1)
    return sec, (SAMPLE_N - 2) * (SAMPLE_N - 2) * iters, used


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    ncores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_sample(1, ncores)
    tot_s, tot_c, used = 0.0, 0, 1
    for _ in range(args.steps):
        s, c, used = oracle_sample(1, ncores)
        tot_s += s
        tot_c += c
    value = tot_c / tot_s / 1e9
    sample = ("%dx%d FP32, 16-device BLOCK partitions, 1 Jacobi iteration per step: per-element "
              "messages (one thread) + value loops (%d threads)" % (SAMPLE_N, SAMPLE_N, used))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_s / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + " (reference: the CPU oracle on a %dx%d sample, one "
                                              "iteration per step)" % (SAMPLE_N, SAMPLE_N)},
            "cpu_baseline": {"kind": "oracle", "cores": used, "nproc": ncores, "value": value, "unit": UNIT,
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------------------
# the other workloads: sub-records of the default line, or one line each with --workload
# ---------------------------------------------------------------------------------------------

def _events(torch, stream, fn, reps):
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _roofline_hbm(kernel, algo_bytes, per_launch_ms, traffic=None):
    pk = peaks()
    ach = algo_bytes / (per_launch_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": pk["hbm"], "unit": "GB/s",
            "frac": ach / pk["hbm"], "peak_source": pk["source"], "traffic": traffic,
            "algo_bytes_per_launch": algo_bytes, "launch_us": per_launch_ms * 1e3}


def _moved(H, arrs, esize):
    import numpy as np
    return sum(int(np.prod(np.subtract(hi, lo))) for a in arrs for _, _, lo, hi in H.HDArrayGetPlan(a)) * esize


def workload_stencil3d(H, torch, stream, args):
    """512^3 binary32 7-point stencil over 37 uneven manual boxes (seeded k-d cuts, extents
    16-256), +-1 faces, 50 iterations per step, one fused launch per iteration (graph)."""
    import numpy as np
    import synthetic
    n, nb, iters = args.n3, args.nb3, 50
    boxes = synthetic.kd_boxes(n, nb, stream=3) if nb > 1 else [((0, 0, 0), (n, n, n))]
    work = [(tuple(max(1, v) for v in lo), tuple(min(n - 1, v) for v in hi)) for lo, hi in boxes]
    x = synthetic.jacobi_field((n, n, n), stream=3, dtype="float")
    xh = torch.from_numpy(x).pin_memory()
    H.HDArrayInit(ndev=nb)
    H.HDArraySetStream(stream.cuda_stream)
    B = H.HDArrayCreate("B", "float", None, n, n, n)
    A = H.HDArrayCreate("A", "float", None, n, n, n)
    D = H.HDArrayPartitionManual((n, n, n), boxes)
    W = H.HDArrayPartitionManual((n, n, n), work)
    H.HDArrayWrite(B, xh, D)
    for _ in range(2):
        H.HDArrayApplyKernel("stencil3d", W, B, A)
        H.HDArrayApplyKernel("stencil3d", W, A, B)
    H.HDArrayApplyKernel("stencil3d", W, B, A)
    xbytes = _moved(H, [B], 4)
    H.HDArrayApplyKernel("stencil3d", W, A, B)
    H.HDArrayGraphBegin()
    H.HDArrayApplyKernel("stencil3d", W, B, A)
    H.HDArrayApplyKernel("stencil3d", W, A, B)
    gid = H.HDArrayGraphEnd()
    for _ in range(args.warmup):
        H.HDArrayGraphLaunch(gid, iters // 2)
    steps = max(2, args.steps)
    ms = _events(torch, stream, lambda: H.HDArrayGraphLaunch(gid, iters // 2), steps)
    cells = sum(int(np.prod(np.subtract(hi, lo))) for lo, hi in work)
    per = ms / iters
    algo = cells * 8 + 2 * xbytes
    parity = None
    if not args.quick:
        # a fresh run of exactly 50 iterations from the input, sampled cells checked
        H.HDArrayWrite(B, xh, D)
        for _ in range(2):
            H.HDArrayApplyKernel("stencil3d", W, B, A)
            H.HDArrayApplyKernel("stencil3d", W, A, B)
        H.HDArrayGraphLaunch(gid, (iters - 4) // 2)
        got = np.zeros((n, n, n), np.float32)
        H.HDArrayRead(B, got, D)
        u = synthetic.uniform(9, stream=903)
        pts = [tuple(1 + int(u[3 * i + d] * (n - 2)) for d in range(3)) for i in range(3)]
        for lo, hi in boxes[:5]:  # cells at box corners: T-junctions of uneven faces
            pts.append(tuple(min(n - 2, max(1, v)) for v in lo))
        parity = cone_check(x, got, pts, iters, np.float32)
    H.HDArrayExit()
    traffic = profiled("stencil3d_cta_fp32_512_37boxes.md", "dram_bytes_per_launch_v%d" % stencil3d_variant(),
                       ["k_stencil3d.cu", "stencil_common.cuh"]) if (n, nb) == (512, 37) else None
    return {"workload": "3-D 7-point %d^3 FP32, %d uneven manual partitions (extents 16-256), +-1 faces, "
                        "50 iterations per step, one fused launch per iteration (graph)" % (n, nb),
            "metric": UNIT, "value": cells * iters / (ms * 1e-3) / 1e9, "unit": UNIT, "dtype": "f32",
            "steps": steps, "ms_per_step": ms, "us_per_iter": per * 1e3,
            "exchange_bytes_per_iteration": 2 * xbytes,
            "roofline": _roofline_hbm({3: "k_stencil3d_tma<f32,8> (planes staged by bulk tensor copies)",
                                       1: "k_stencil3d_cta<f32,8> (cp.async plane ring)"}.get(
                                          stencil3d_variant(), "k_stencil3d") + ", fused exchange + stencil",
                                      algo, per, traffic),
            "parity": parity}


def workload_conv2d(H, torch, stream, args):
    """The 2-D convolution of Sec. 5 (eight neighbours and the centre, seeded weights) on the
    8192^2 binary32 grid, BLOCK 4 x 4; no dependency between iterations, so the halo moves once."""
    import synthetic
    N, P, iters = args.grid, 16, 100
    x = synthetic.jacobi_field((N, N), stream=6, dtype="float")
    w = [float(v) for v in synthetic.normal(9, stream=6)]
    H.HDArrayInit(ndev=P)
    H.HDArraySetStream(stream.cuda_stream)
    X = H.HDArrayCreate("X", "float", None, N, N)
    Y = H.HDArrayCreate("Y", "float", None, N, N)
    D = H.HDArrayPartition(H.BLOCK, (N, N), (0, 0), (N, N), P)
    W = H.HDArrayPartition(H.BLOCK, (N, N), (1, 1), (N - 1, N - 1), P)
    H.HDArrayWrite(X, torch.from_numpy(x).pin_memory(), D)
    for _ in range(2):
        H.HDArrayApplyKernel("conv2d", W, X, Y, *w)
    H.HDArrayGraphBegin()
    H.HDArrayApplyKernel("conv2d", W, X, Y, *w)
    H.HDArrayApplyKernel("conv2d", W, X, Y, *w)
    gid = H.HDArrayGraphEnd()
    for _ in range(args.warmup):
        H.HDArrayGraphLaunch(gid, iters // 2)
    ms = _events(torch, stream, lambda: H.HDArrayGraphLaunch(gid, iters // 2), args.steps)
    cells = (N - 2) * (N - 2)
    per = ms / iters
    H.HDArrayExit()
    return {"workload": "2-D convolution (3 x 3 weights) %d^2 FP32, BLOCK 4x4 = 16 logical devices, "
                        "%d iterations per step" % (N, iters),
            "metric": UNIT, "value": cells * iters / (ms * 1e-3) / 1e9, "unit": UNIT,
            "ms_per_step": ms, "us_per_iter": per * 1e3,
            "roofline": _roofline_hbm("k_jacobi2d_tma<f32,4,4,OP_CONV> (rows staged by bulk tensor copies)"
                                      if conv_variant() == 5 else "k_jacobi2d_cta<f32,8,OP_CONV> (packed row streams)",
                                      cells * 8, per)}


def workload_2mm(H, torch, stream, args):
    """2MM (Sec. 5.1): D = A B, then E = C D, every iteration, on 8 logical devices with row
    blocks and with column blocks -- the same products, different exchanges (Table 3's
    partitioning study).  binary32 arrays on the tensor cores (bf16x3)."""
    import synthetic
    n, P, iters = args.n2mm, 8, 4
    host = {x: torch.from_numpy(synthetic.to_storage(synthetic.normal(n * n, stream=7 * 10 + i).reshape(n, n),
                                                      "float")).pin_memory() for i, x in enumerate("ABCDE")}
    flops = 2 * 2.0 * n * n * n  # two products per iteration
    forms = {}
    for form, ptype in (("row", H.ROW), ("col", H.COL)):
        H.HDArrayInit(ndev=P)
        H.HDArraySetStream(stream.cuda_stream)
        arr = {x: H.HDArrayCreate(x, "float", None, n, n) for x in "ABCDE"}
        Q = H.HDArrayPartition(ptype, (n, n), (0, 0), (n, n), P)
        for x in "ABCDE":
            H.HDArrayWrite(arr[x], host[x], Q)

        def iteration():
            H.HDArrayApplyKernel("gemm", Q, arr["A"], arr["B"], arr["D"], 1.0, 0.0, n, n, n)
            moved = _moved(H, [arr["A"], arr["B"]], 4)
            H.HDArrayApplyKernel("gemm", Q, arr["C"], arr["D"], arr["E"], 1.0, 0.0, n, n, n)
            return moved + _moved(H, [arr["C"], arr["D"]], 4)

        first = iteration()
        steady = iteration()
        H.HDArrayGraphBegin()
        iteration()
        gid = H.HDArrayGraphEnd()
        for _ in range(args.warmup):
            H.HDArrayGraphLaunch(gid, iters)
        ms = _events(torch, stream, lambda: H.HDArrayGraphLaunch(gid, iters), args.steps)
        per = ms / iters
        forms[form] = {"ms_per_iteration": per, "tflops_algorithmic": flops / (per * 1e-3) / 1e12,
                       "exchange_bytes_first_iteration": first, "exchange_bytes_per_iteration": steady}
        H.HDArrayExit()
    peak = peaks()["bf16"]
    best = forms["col"]
    return {"workload": "2MM (D = A B, E = C D) %d^2 FP32 on tensor cores (bf16x3), 8 logical devices, "
                        "row vs column blocks, %d iterations per step" % (n, iters),
            "metric": "TFLOP/s (algorithmic)", "value": best["tflops_algorithmic"],
            "ms_per_step": best["ms_per_iteration"] * iters, "forms": forms,
            "roofline": {"bound": "tensor", "kernel": "bf16x3 tcgen05 GEMM",
                         "achieved": 3 * best["tflops_algorithmic"], "peak": peak, "unit": "TFLOP/s",
                         "frac": 3 * best["tflops_algorithmic"] / peak,
                         "note": "issued MMA flops (3 products per bf16x3 step) of the column form"}}


def workload_cov(H, torch, stream, args):
    """Covariance (Sec. 5.1) of n samples x m variables, binary32 (the product on the tensor
    cores, bf16x3), 32 logical devices: column means, centring, the upper-triangular product with
    absolute use / trapezoid definition sections, the symmetric copy.  Row blocks of C split
    evenly and balanced by the upper triangle's area (a manual partition)."""
    import synthetic
    from paper_1809_05657_gb300.partitions import even_rows, triangle_balanced_rows as balanced_rows
    n = m = args.ncov
    P, iters = 32, 2
    x = torch.from_numpy(synthetic.to_storage(synthetic.normal(n * m, stream=8).reshape(n, m), "float")).pin_memory()
    flops = float(n) * m * (m + 1)  # the product's upper triangle (j >= i)
    forms = {}
    for form in ("even", "balanced"):
        rows = balanced_rows(m, P) if form == "balanced" else even_rows(m, P)
        H.HDArrayInit(ndev=P)
        H.HDArraySetStream(stream.cuda_stream)
        X = H.HDArrayCreate("X", "float", None, n, m)
        M = H.HDArrayCreate("M", "float", None, 1, m)
        Xc = H.HDArrayCreate("Xc", "float", None, n, m)
        C = H.HDArrayCreate("C", "float", None, m, m)
        DX = H.HDArrayPartition(H.ROW, (n, m), (0, 0), (n, m), P)
        PM = H.HDArrayPartition(H.COL, (1, m), (0, 0), (1, m), P)
        PC = H.HDArrayPartitionManual((m, m), [((rows[p], 0), (rows[p + 1], m)) for p in range(P)])
        for p in range(P):
            r0, r1 = rows[p], rows[p + 1]
            H.HDArraySetAbsoluteUse("syrk", PC, Xc, p, (0, r0), (n, m))
            H.HDArraySetTrapezoidDef("syrk", PC, C, p, (r0, r0, r0, m - 1, r1 - 1, r1 - 1, r1 - 1, m - 1))
            H.HDArraySetAbsoluteUse("symmetrize", PC, C, p, (0, r0), (r1, r1))
            t = max(r0, 1)
            if t < r1:
                H.HDArraySetTrapezoidDef("symmetrize", PC, C, p, (t, 0, t, t - 1, r1 - 1, 0, r1 - 1, r1 - 2))
            else:
                H.HDArraySetAbsoluteDef("symmetrize", PC, C, p, (0, 0), (0, 0))
        H.HDArrayWrite(X, x, DX)

        def iteration():
            v = 0
            H.HDArrayApplyKernel("colmean", PM, X, M)
            v += _moved(H, [X], 4)
            H.HDArrayApplyKernel("center", DX, X, M, Xc)
            v += _moved(H, [X, M], 4)
            H.HDArrayApplyKernel("syrk", PC, Xc, C, 1.0 / (n - 1))
            v += _moved(H, [Xc], 4)
            H.HDArrayApplyKernel("symmetrize", PC, C)
            v += _moved(H, [C], 4)
            return v

        first = iteration()
        steady = iteration()
        H.HDArrayGraphBegin()
        iteration()
        gid = H.HDArrayGraphEnd()
        for _ in range(args.warmup):
            H.HDArrayGraphLaunch(gid, iters)
        ms = _events(torch, stream, lambda: H.HDArrayGraphLaunch(gid, iters), args.steps)
        per = ms / iters
        forms[form] = {"ms_per_iteration": per, "tflops_algorithmic": flops / (per * 1e-3) / 1e12,
                       "exchange_bytes_first_iteration": first, "exchange_bytes_per_iteration": steady,
                       "row_bounds_head": rows[:4]}
        H.HDArrayExit()
    best = min(forms.values(), key=lambda f: f["ms_per_iteration"])
    return {"workload": "covariance of %d samples x %d variables, FP32 (product on tensor cores, bf16x3), "
                        "32 logical devices, even vs area-balanced row blocks, %d iterations per step" % (n, m, iters),
            "metric": "TFLOP/s (algorithmic, the product's upper triangle)", "value": best["tflops_algorithmic"],
            "ms_per_step": best["ms_per_iteration"] * iters, "forms": forms}


def workload_small(H, torch, stream, args):
    """The 256^2 binary64 Jacobi of the paper's program (ROW 4, 10 iterations) and the FP64
    residual via HDArrayReduce: it fits in L2 and is bound by launch latency, so it reports
    microseconds per iteration, no roofline claim.  Plain form: the paper's two kernels (the step,
    then the copy back), one launch per device and kernel, no graph.  Fused form: the step alone
    with the arrays' roles swapped every iteration (the same values and messages), one launch per
    iteration, the 10 iterations replayed as a CUDA graph.  Both end with the residual of the last
    iteration, sum((new - old)^2), folded in different orders (a separate reduction launch in the
    plain form, the residual launch's own fold in the fused form), so they agree to the reduction
    bound; the final field (bit for bit) and the residual are checked against a numpy binary64
    evaluation of the same number of iterations."""
    import numpy as np
    import synthetic
    N, P, iters = 256, 4, 10
    x = synthetic.jacobi_field((N, N), stream=0, dtype="double")
    out = {}
    steps = max(2, args.steps)
    for form, mode in (("plain", H.HDARRAY_MODE_PLAIN), ("fused", H.HDARRAY_MODE_FUSED)):
        H.HDArrayInit(ndev=P)
        H.HDArraySetStream(stream.cuda_stream)
        H.HDArraySetMode(mode)
        B = H.HDArrayCreate("B", "double", None, N, N)
        A = H.HDArrayCreate("A", "double", None, N, N)
        R = H.HDArrayCreate("R", "double", None, N, N)
        D = H.HDArrayPartition(H.ROW, (N, N), (0, 0), (N, N), P)
        W = H.HDArrayPartition(H.ROW, (N, N), (1, 1), (N - 1, N - 1), P)

        H.HDArrayWrite(B, x, D)
        H.HDArrayWrite(A, x, D)
        setup = 6  # iterations before the timed steps, the same in both forms
        if form == "plain":
            for _ in range(setup):
                H.HDArrayApplyKernel("jacobi2d", W, B, A)
                H.HDArrayApplyKernel("copy", W, A, B)

            def step():
                for _ in range(iters - 1):
                    H.HDArrayApplyKernel("jacobi2d", W, B, A)
                    H.HDArrayApplyKernel("copy", W, A, B)
                H.HDArrayApplyKernel("jacobi2d", W, B, A)
                H.HDArrayApplyKernel("sqdiff", W, A, B, R)   # new iterate A against the old B
                r = H.HDArrayReduce(R, H.SUM, W)
                H.HDArrayApplyKernel("copy", W, A, B)
                return r
        else:
            for _ in range(2):  # plans and buffers settle before the recording
                H.HDArrayApplyKernel("jacobi2d", W, B, A)
                H.HDArrayApplyKernel("jacobi2d", W, A, B)
            H.HDArrayGraphBegin()
            H.HDArrayApplyKernel("jacobi2d", W, B, A)
            H.HDArrayApplyKernel("jacobi2d", W, A, B)
            gid = H.HDArrayGraphEnd()  # recording also ran its two iterations: 6 in all

            def step():  # 10 iterations end with the new iterate in B, the old in A
                H.HDArrayGraphLaunch(gid, iters // 2)
                H.HDArrayApplyKernel("sqdiff", W, B, A, R)
                return H.HDArrayReduce(R, H.SUM, W)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            res = step()
        dt = (time.perf_counter() - t0) / steps
        res_iters = setup + (args.warmup + steps) * iters  # the last residual's iteration
        out[form] = {"ms_per_step": dt * 1e3, "us_per_iteration": dt * 1e6 / iters, "residual": res}
        if form == "fused":  # the iterations alone, on the device (the graph replays, no residual)
            out[form]["device_us_per_iteration"] = _events(
                torch, stream, lambda: H.HDArrayGraphLaunch(gid, iters // 2), steps) * 1e3 / iters
            field_iters = res_iters + steps * iters
            got = np.zeros((N, N), np.float64)
            H.HDArrayRead(B, got, D)  # a use by the data partition: after the last graph replay
        H.HDArrayExit()
    # numpy binary64 evaluation of the same iterations and the last residual
    prev = stencil_steps(x, res_iters - 1, np.float64)
    last = stencil_steps(prev, 1, np.float64)
    res_ref = float(np.sum((last[1:-1, 1:-1] - prev[1:-1, 1:-1]) ** 2))
    field = stencil_steps(last, field_iters - res_iters, np.float64)
    cells = (N - 2) * (N - 2)
    best = out["fused"]
    return {"workload": "Jacobi 256^2 FP64, ROW 4 = 4 logical devices, 10 iterations + FP64 residual "
                        "(HDArrayReduce, synchronous) per step; host wall clock per step (plain: the paper's "
                        "step and copy kernels; fused: the step with roles swapped, in a graph)",
            "metric": UNIT, "value": cells * iters / (best["ms_per_step"] * 1e-3) / 1e9, "unit": UNIT,
            "dtype": "f64", "steps": steps, "ms_per_step": best["ms_per_step"], "forms": out,
            "parity": {"residual_rel_diff_plain_fused": abs(out["plain"]["residual"] - out["fused"]["residual"])
                                                        / abs(out["fused"]["residual"]),
                       "field_bit_exact_vs_numpy_binary64": bool(np.array_equal(got, field)),
                       "residual_rel_err_vs_numpy": abs(best["residual"] - res_ref) / abs(res_ref),
                       "iterations": field_iters},
            "roofline": {"bound": "launch latency", "note": "fits in L2; reported in microseconds per iteration",
                         "frac": None}}


def workload_batch(H, torch, stream, args):
    """512 independent Jacobi instances (sides log-uniform 64..2048, 2-16 ROW/COL partitions each,
    binary32), all instances' exchanges and stencils in one launch per iteration (a batch),
    200 iterations per step replayed from a graph."""
    import numpy as np
    import synthetic
    insts = synthetic.jacobi_instances(args.ninst, stream=5)
    iters = 200
    ndev = max(p for _, _, p, _ in insts)
    H.HDArrayInit(ndev=ndev)
    H.HDArraySetStream(stream.cuda_stream)
    arrs = []
    cells = 0
    for i, (r, c, P, kind) in enumerate(insts):
        t = H.ROW if kind == "ROW" else H.COL
        x = synthetic.jacobi_field((r, c), stream=1000 + i, dtype="float")
        B = H.HDArrayCreate("B", "float", None, r, c)
        A = H.HDArrayCreate("A", "float", None, r, c)
        D = H.HDArrayPartition(t, (r, c), (0, 0), (r, c), P)
        W = H.HDArrayPartition(t, (r, c), (1, 1), (r - 1, c - 1), P)
        H.HDArrayWrite(B, x, D)
        arrs.append((B, A, W, D))
        cells += (r - 2) * (c - 2)

    def iteration(flip):
        H.HDArrayBatchBegin()
        for B, A, W, _ in arrs:
            if flip:
                H.HDArrayApplyKernel("jacobi2d", W, A, B)
            else:
                H.HDArrayApplyKernel("jacobi2d", W, B, A)
        H.HDArrayBatchEnd()

    xbytes = 0
    for k in range(2):
        iteration(False)
        if k == 1:
            xbytes = _moved(H, [B for B, _, _, _ in arrs], 4)
        iteration(True)
    H.HDArrayGraphBegin()
    iteration(False)
    iteration(True)
    gid = H.HDArrayGraphEnd()
    for _ in range(args.warmup):
        H.HDArrayGraphLaunch(gid, iters // 2)
    steps = max(2, args.steps)
    ms = _events(torch, stream, lambda: H.HDArrayGraphLaunch(gid, iters // 2), steps)
    per = ms / iters
    total_iters = 6 + (args.warmup + steps) * iters
    parity = None
    if not args.quick:
        # the three smallest instances against a numpy binary32 evaluation of every iteration
        small = sorted(range(len(insts)), key=lambda i: insts[i][0] * insts[i][1])[:3]
        exact = 0
        for i in small:
            r, c, _, _ = insts[i]
            B, A, W, D = arrs[i]
            got = np.zeros((r, c), np.float32)
            H.HDArrayRead(B, got, D)
            ref = stencil_steps(synthetic.jacobi_field((r, c), stream=1000 + i, dtype="float"), total_iters, np.float32)
            exact += int(np.array_equal(got.view(np.uint32), ref.view(np.uint32)))
        parity = {"instances_checked": len(small), "bit_exact_binary32": exact, "iterations": total_iters,
                  "shapes": [list(insts[i]) for i in small], "reference": "numpy binary32, every iteration"}
    H.HDArrayExit()
    traffic = profiled("jacobi2d_batch512_fp32.md", "dram_bytes_per_launch",
                       ["k_stencil2d.cu", "stencil_common.cuh"]) if args.ninst == 512 else None
    return {"workload": "batch of %d Jacobi instances (sides log-uniform 64..2048, 2-16 ROW/COL partitions "
                        "each, FP32), all instances in one launch per iteration, 200 iterations per step "
                        "(graph)" % len(insts),
            "metric": UNIT, "value": cells * iters / (ms * 1e-3) / 1e9, "unit": UNIT, "dtype": "f32",
            "cells": cells, "steps": steps, "ms_per_step": ms, "us_per_iter": per * 1e3,
            "exchange_bytes_per_iteration": 2 * xbytes,
            "roofline": _roofline_hbm("k_jacobi2d (batched, fused exchange)", cells * 8 + 2 * xbytes, per, traffic),
            "parity": parity}


def fp64_peak(torch):
    """Measured FP64 matrix-multiply rate of this GPU: cuBLAS DGEMM (torch.matmul) 8192^3,
    best of 5.  The denominator of the DFMA GEMM's fraction."""
    a = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    b = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * 8192 ** 3 / (best * 1e-3) / 1e12


def workload_trmm(H, torch, stream, args):
    """tril(A) 8192 x 8192 times B 8192 x 4096 over 8 row partitions (trapezoid use of A, B used
    whole): the binary64 form (DFMA), and binary32 arrays on the bf16 tensor cores in the bf16x6
    form (three-way split, meets the binary32 accuracy bound componentwise; the value) and the
    bf16x3 form; the all-gather of B alone."""
    import numpy as np
    import synthetic
    n, m, P = 8192, 4096, 8
    a, b = synthetic.tri_gemm_inputs(n, m, stream=4, dtype="double")
    pk = peaks()
    H.HDArrayInit(ndev=P)
    H.HDArraySetStream(stream.cuda_stream)
    A = H.HDArrayCreate("A", "double", None, n, n)
    B = H.HDArrayCreate("B", "double", None, n, m)
    C = H.HDArrayCreate("C", "double", None, n, m)
    R = H.HDArrayPartition(H.ROW, (n, m), (0, 0), (n, m), P)
    RA = H.HDArrayPartition(H.ROW, (n, n), (0, 0), (n, n), P)
    rows = [n * p // P for p in range(P + 1)]
    for p in range(P):
        r0, r1 = rows[p], rows[p + 1]
        H.HDArraySetTrapezoidUse("trmm", R, A, p, (r0, 0, r0, r0, r1 - 1, 0, r1 - 1, r1 - 1))
        H.HDArraySetAbsoluteUse("exchange", R, B, p, (0, 0), (n, m))
    bh = torch.from_numpy(b).pin_memory()
    H.HDArrayWrite(A, torch.from_numpy(a).pin_memory(), RA)
    # the all-gather of B alone (7/8 of B to each of 8 devices), timed from freshly written B
    ex = []
    for _ in range(max(3, args.steps // 4)):
        H.HDArrayWrite(B, bh, R)
        ex.append(_events(torch, stream, lambda: H.HDArrayApplyKernel("exchange", R, B), 1))
    moved = 7 * n * m * 8
    exch_ms = statistics.median(ex[1:])
    H.HDArrayWrite(B, bh, R)
    H.HDArrayApplyKernel("trmm", R, A, B, C, 1.0, 0.0)  # first call carries the all-gather
    H.HDArrayApplyKernel("trmm", R, A, B, C, 1.0, 0.0)
    reps64 = max(2, args.steps // 8)
    ms = _events(torch, stream, lambda: H.HDArrayApplyKernel("trmm", R, A, B, C, 1.0, 0.0), reps64)
    flops = 2.0 * m * (n * (n + 1) / 2)
    H.HDArrayExit()
    f64peak = fp64_peak(torch)
    out = {"workload": "tril(A) 8192x8192 x B 8192x4096 (N(0,1)), 8 row partitions with trapezoid use of A, "
                       "B used whole (all-gather once); FP32 arrays on BF16 tensor cores (bf16x6 = the value, "
                       "bf16x3) and the FP64 plain form (DFMA)",
           "metric": "TFLOP/s (algorithmic)", "unit": "TFLOP/s",
           "fp64": {"tflops_algorithmic": flops / (ms * 1e-3) / 1e12, "ms_per_call": ms, "calls": reps64,
                    "roofline": {"bound": "fp64", "achieved": flops / (ms * 1e-3) / 1e12, "peak": f64peak,
                                 "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / 1e12 / f64peak,
                                 "peak_source": "measured in this run: cuBLAS DGEMM 8192^3 (torch.matmul)",
                                 "frac_of_nominal": flops / (ms * 1e-3) / 1e12 / 1.25,
                                 "nominal": "1.25 TFLOP/s FP64 (GB300 data sheet)"}},
           "exchange": {"bytes": moved, "ms": exch_ms, "GB_s": 2 * moved / (exch_ms * 1e-3) / 1e9,
                        "hbm_frac": 2 * moved / (exch_ms * 1e-3) / 1e9 / pk["hbm"], "peak_source": pk["source"]}}
    out["bf16x6"] = trmm_tc(H, torch, stream, args, a, b, 3)
    out["bf16x3"] = trmm_tc(H, torch, stream, args, a, b, 2)
    x6 = out["bf16x6"]
    out["value"] = x6["tflops_algorithmic"]
    out["ms_per_step"] = x6["ms_per_call"]
    out["steps"] = x6["calls"]
    out["dtype"] = "bf16 (x6 split of f32)"
    traffic = None
    out["roofline"] = {"bound": "tensor", "kernel": "k_gemm_bf16x3_panels<3> (bf16x6, tcgen05)",
                       "achieved": x6["tflops_mma_issued"], "peak": pk["bf16"], "unit": "TFLOP/s",
                       "frac": x6["tflops_mma_issued"] / pk["bf16"], "peak_source": pk["source"],
                       "traffic": traffic, "frac_algorithmic": x6["tflops_algorithmic"] / pk["bf16"],
                       "note": "achieved counts issued MMA flops (6 products per K step over whole tiles); "
                               "frac_algorithmic counts the triangle's 2.75e11 flops once"}
    return out


def trmm_tc(H, torch, stream, args, a64, b64, split):
    """The triangular product on binary32 arrays on the tensor cores, in the bf16x3 (split 2) or
    bf16x6 (split 3) form.  Times the call with its operands' split panels reused (A and B
    unchanged) and, separately, the call right after B was rewritten (B's all-gather to the eight
    devices and the re-split of its panels included); the
    componentwise error against a numpy binary64 product of the binary32 inputs on sampled
    entries, among them the first rows, where few terms leave the split's error unaveraged."""
    import numpy as np
    n, m, P = 8192, 4096, 8
    a = a64.astype(np.float32)
    b = b64.astype(np.float32)
    H.HDArrayInit(ndev=P)
    H.HDArraySetStream(stream.cuda_stream)
    H.HDArraySetGemmSplit(split)
    A = H.HDArrayCreate("A", "float", None, n, n)
    B = H.HDArrayCreate("B", "float", None, n, m)
    C = H.HDArrayCreate("C", "float", None, n, m)
    R = H.HDArrayPartition(H.ROW, (n, m), (0, 0), (n, m), P)
    RA = H.HDArrayPartition(H.ROW, (n, n), (0, 0), (n, n), P)
    for p in range(P):
        r0, r1 = n * p // P, n * (p + 1) // P
        H.HDArraySetTrapezoidUse("trmm", R, A, p, (r0, 0, r0, r0, r1 - 1, 0, r1 - 1, r1 - 1))
    bh = torch.from_numpy(b).pin_memory()
    H.HDArrayWrite(A, torch.from_numpy(a).pin_memory(), RA)
    H.HDArrayWrite(B, bh, R)
    H.HDArrayApplyKernel("trmm", R, A, B, C, 1.0, 0.0)
    for _ in range(args.warmup):
        H.HDArrayApplyKernel("trmm", R, A, B, C, 1.0, 0.0)
    reps = max(2, args.steps)
    ms = _events(torch, stream, lambda: H.HDArrayApplyKernel("trmm", R, A, B, C, 1.0, 0.0), reps)
    after_write = []
    for _ in range(3):  # B rewritten: the call all-gathers B again and re-splits its panels
        H.HDArrayWrite(B, bh, R)  # (the host copy itself finishes before the timing starts)
        after_write.append(_events(torch, stream, lambda: H.HDArrayApplyKernel("trmm", R, A, B, C, 1.0, 0.0), 1))
    got = np.zeros((n, m), np.float32)
    H.HDArrayRead(C, got, R)
    H.HDArrayExit()
    rng = np.random.default_rng(4)
    ij = np.stack([rng.integers(0, n, 256), rng.integers(0, m, 256)], 1)
    ij = np.concatenate([ij, [[0, 0], [1, 5], [127, 4095], [128, 1], [8191, 4095], [4095, 2048]],
                         [[i, j] for i in range(4) for j in rng.integers(0, m, 64)]])
    a64f, b64f = a.astype(np.float64), b.astype(np.float64)
    ref = np.array([a64f[i, :i + 1] @ b64f[:i + 1, j] for i, j in ij])
    mag = np.array([np.abs(a64f[i, :i + 1]) @ np.abs(b64f[:i + 1, j]) for i, j in ij])
    g = got[ij[:, 0], ij[:, 1]].astype(np.float64)
    flops = 2.0 * m * (n * (n + 1) / 2)
    products = 3 if split == 2 else 6
    issued = 0.0  # MMA flops actually issued: 3 or 6 products per K step over whole 128-row tiles
    for ti in range(0, n, 128):
        kend = min(n, ti + 128)
        issued += products * 2.0 * 128 * m * ((kend + 63) // 64 * 64)
    peak = peaks()["bf16"]
    rewrite_ms = statistics.median(after_write) - ms
    return {"ms_per_call": ms, "calls": reps, "tflops_algorithmic": flops / (ms * 1e-3) / 1e12,
            "tflops_mma_issued": issued / (ms * 1e-3) / 1e12,
            "tensor_frac": issued / (ms * 1e-3) / 1e12 / peak, "peak_tflops": peak,
            "ms_per_call_after_b_write": statistics.median(after_write),
            "b_allgather_and_split_ms": rewrite_ms,
            "err_componentwise_max": float((np.abs(g - ref) / mag).max()),
            "err_normwise": float(np.abs(g - ref).max() / np.abs(ref).max()),
            "samples": int(len(ij)), "products_per_k_step": products,
            "reference": "numpy binary64 dot products of the binary32 inputs"}


WORKLOADS = {"stencil3d": workload_stencil3d, "batch": workload_batch, "trmm": workload_trmm,
             "conv2d": workload_conv2d, "2mm": workload_2mm, "cov": workload_cov, "small": workload_small}
# the default line's sub-records: the workloads the benchmark's configurations name
DEFAULT_SUB = [("jacobi2d_256_fp64_row4", "small"), ("stencil3d_512_fp32_37boxes", "stencil3d"),
               ("trmm_8192x4096_8parts", "trmm"), ("batch512_jacobi2d_fp32", "batch")]


def run_workload(args):
    import torch
    from __graft_entry__ import build_library
    from paper_1809_05657_gb300 import hdarray as H
    build_library()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    tpath = tune_setup(args)
    out = WORKLOADS[args.workload](H, torch, stream, args)
    out["autotuned"] = tune_report(tpath)
    out["steps"] = out.get("steps", args.steps)
    out["warmup"] = args.warmup
    print(json.dumps(out))
    return 0


def sub_workloads(args):
    """The other workloads as sub-records of the default line (each on its own context)."""
    import torch
    from paper_1809_05657_gb300 import hdarray as H
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {}
    for key, name in DEFAULT_SUB:
        t = time.perf_counter()
        try:
            r = WORKLOADS[name](H, torch, stream, args)
        except Exception as e:  # a failing sub-workload is reported, the headline still prints
            r = {"error": "%s: %s" % (type(e).__name__, e)}
            try:
                H.HDArrayExit()
            except Exception:
                pass
        r["wall_s"] = time.perf_counter() - t
        out[key] = r
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--quick", action="store_true",
                    help="headline only: skip the comparison forms, e2e, parity checks and sub-records")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="use the default tile shapes")
    ap.add_argument("--storage", default="float", choices=["float", "bf16"],
                    help="headline workload's storage type (bf16 for profiling the BF16 form alone)")
    ap.add_argument("--grid", type=int, default=8192,
                    help="grid side (default 8192; smaller only for profiling captures)")
    ap.add_argument("--n3", type=int, default=512, help="3-D workload: cube side")
    ap.add_argument("--nb3", type=int, default=37, help="3-D workload: number of boxes (1 = one box)")
    ap.add_argument("--ninst", type=int, default=512, help="batch workload: number of instances")
    ap.add_argument("--n2mm", type=int, default=8192, help="2mm workload: matrix side")
    ap.add_argument("--ncov", type=int, default=10240, help="cov workload: samples = variables")
    ap.add_argument("--workload", default="jacobi2d",
                    choices=["jacobi2d", "stencil3d", "batch", "trmm", "conv2d", "2mm", "cov", "small"],
                    help="jacobi2d is the benchmark line; the others print their own line")
    args = ap.parse_args()
    global N, CELLS
    N = args.grid
    CELLS = (N - 2) * (N - 2)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.workload != "jacobi2d":
        return run_workload(args)
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    tpath = tune_setup(args)
    r = gpu_arm(args, rank, world)
    tuned = tune_report(tpath)
    subs = None
    if rank == 0 and not args.quick and args.storage == "float":
        subs = sub_workloads(args)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    if rank == 0:
        variant = jacobi_variant(tuned, "f32" if args.storage == "float" else "bf16")
        traffic = profiled("jacobi2d_fp32_8192_block16.md", "dram_bytes_per_launch_v%d" % variant,
                           ["k_stencil2d.cu", "stencil_common.cuh"]) if N == 8192 and args.storage == "float" else None
        pk = r["peaks"]
        line = {
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.storage == "float" else "bf16 storage, f32 arithmetic",
            "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("8192x8192", "%dx%d" % (N, N)).replace(
                           "FP32", "FP32" if args.storage == "float" else "BF16 storage"),
                       "grid": [N, N], "logical_devices": P,
                       "iterations_per_step": ITERS, "parallelism": "replicas" if world > 1 else "1 GPU",
                       "l2": "inputs 2 x %d MiB %s 129 MB L2 (no flush)" % (N * N * 4 // 2 ** 20, ">" if N * N * 4 > 129e6 else "<=")},
            "roofline": {"bound": "hbm", "kernel": KERNEL_NAMES_2D[variant].replace("f32", "f32" if args.storage == "float" else "bf16") + ", fused exchange + stencil",
                         "achieved": r["achieved"], "peak": pk["hbm"], "unit": "GB/s",
                         "frac": r["achieved"] / pk["hbm"], "peak_source": pk["source"],
                         "traffic": traffic, "algo_bytes_per_launch": r["algo_bytes"],
                         "launch_us": r["per_launch_ms"] * 1e3},
            "exchange": {"bytes_per_iteration": r["xbytes"] * 2, "note": "halo read+write, fused"},
            "residual_us_per_step": r["residual_us"],
            "cpu_baseline": cpu,
            "e2e": r["e2e"],
            "gpu_launches": r["launches"],
            "clocks": r["clocks"],
            "residual": r["residual"],
            "parity": r["parity"],
            "autotuned": tuned,
            "forms": r["extra"],
            "workloads": subs,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
