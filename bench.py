#!/usr/bin/env python
"""Throughput of the rational-function log-det estimator on one GB300.

One step = one complete estimate of log det M for the workload
``matern_n1048576_d4`` (n = 2^20 points uniform in [0,1]^4, Matern-5/2,
lengthscale 0.1, variance 1, noise 1e-2, r_3, rank-512 randomized-SVD
preconditioner with 2 subspace iterations, 16 Rademacher probes, t = 20
Lanczos/CG steps as in Section 3, plus the fp64-normed residual check):
preconditioner build + Algorithm 1, inputs resident in HBM.

Prints one JSON line (metric: log det estimates/s).  --impl reference times
the CPU FP64 oracle on the host cores on a bounded sample of the same
workload instead.  Multi-GPU (torchrun): every rank runs its own independent
estimate (different probe seed), no collective on the data path; value is the
total over ranks ("weak" scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "matern_n1048576_d4"
METRIC = "log det estimates/sec at n=2^20 (Matern-5/2, d=4, r_3, rank 512, 16 probes, t=20)"
UNIT = "estimates/s"

# GB300 ALU roofline for the kernel product: per SM and
# clock, 128 fp32 lane-ops, 32 MUFU ex2 and 16 MUFU sqrt; 152 SMs at 2070 MHz.
# Algorithmic work per pair (i, j): Matern-5/2 d coordinate differences and
# squares, two FMAs of the polynomial and one product (2d + 3 fp32 ops), one
# sqrt and one ex2; RBF 2d fp32 ops and one ex2.
SMS, SM_MHZ_MAX, FP32_PER_CLK, EX2_PER_CLK, SQRT_PER_CLK = 152, 2070.0, 128, 32, 16

# rows of the matrix-free oracle product sampled per host core, in both the
# cpu_baseline leg and the --impl reference arm
ROWS_PER_CORE = 4


# DRAM traffic of one launch of the dominant kernel (ncu dram__bytes_read.sum +
# dram__bytes_write.sum, one pass, n = 2^20, 16 columns, hi/lo fp16: 1.04 GB read +
# 0.74 GB written), valid only for the kernel sources it was taken on (first 16 hex
# digits of their sha256); reported as null once those sources change.
KZ_SYM_TRAFFIC = {"bytes": 640137216 + 523443200,
                  "sources": {"paper_2405_03474_gb300/csrc/kz_sym.cu": "ffc1f6ce5f92d978",
                              "paper_2405_03474_gb300/csrc/point_order.cu": "4fec982c8b04b2a4",
                              "paper_2405_03474_gb300/csrc/tc_common.cuh": "9ab49c92642e95a3"}}


def measured_traffic(record):
    import hashlib
    for rel, digest in record["sources"].items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != digest:
                return None
    return record["bytes"]


def pair_peak_gps(kind, d):
    """Peak kernel-pair evaluations per second (Gpair/s) of the ALU roofline."""
    if kind == "matern52":
        fp32, mufu_clk = 2 * d + 3, 1.0 / SQRT_PER_CLK + 1.0 / EX2_PER_CLK
    else:
        fp32, mufu_clk = 2 * d, 1.0 / EX2_PER_CLK
    per_clk = min(FP32_PER_CLK / fp32, 1.0 / mufu_clk)
    return SMS * per_clk * SM_MHZ_MAX * 1e6 / 1e9


def rank_probe_seed(rank):
    """Probe seed of one rank: every rank estimates with probes of its own, so the
    ranks' estimates are independent units of work (no data-path collective)."""
    from paper_2405_03474_gb300 import inputs
    return inputs.SEED_PROBES + 1000 * rank


def max_over_ranks(ms, world, device):
    """The slowest rank's time: the job ends when its last rank ends."""
    if world == 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, ms_max):
    """Whole-job throughput: every rank completes `steps` estimates in ms_max."""
    return world * steps / (ms_max / 1e3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f16x3_tc")
    ap.add_argument("--sketch-precision", default="f16_tc")
    ap.add_argument("--t", type=int, default=20)
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-precision-compare", action="store_true",
                    help="skip the one-launch-per-precision product comparison after the timed region")
    ap.add_argument("--estimate-compare", default="fp32", metavar="PRECS",
                    help="comma-separated precisions whose estimate is run once after the timed region with the "
                         "same preconditioner and probes ('' to skip; fp64 imports the preconditioner's factors "
                         "into an FP64 handle)")
    ap.add_argument("--no-grad-side", action="store_true",
                    help="skip the gradient side line (logdet_grad on the 2^17-point gradient workload)")
    ap.add_argument("--dense-only", type=int, default=0, metavar="N",
                    help="profiling aid: the stored-M tensor-core product (hi/lo fp16, 64 columns) on N points of "
                         "the stored-dense workload (2 warm-up + 1 launch)")
    ap.add_argument("--cg-only", action="store_true",
                    help="profiling aid: one estimate at --n with a rank-64 preconditioner and 2 CG steps (the CG "
                         "vector updates and preconditioner applies at full vector size)")
    ap.add_argument("--kz-only", type=int, default=0, metavar="C",
                    help="profiling aid: run only the kernel product on C columns (2 warm-up + 1 launch)")
    return ap.parse_args()


def config_of(args, w):
    """The workload's configuration, the same in both arms' JSON lines."""
    from paper_2405_03474_gb300 import inputs
    return {"workload": WORKLOAD, "n": w["n"], "d": w["d"],
            "kernel": "matern52" if w["kind"] == inputs.MATERN52 else "rbf", "lengthscale": w["lengthscale"],
            "variance": w["variance"], "noise": w["noise"], "order": w["order"], "rank": w["rank"],
            "power_iters": w["power_iters"], "probes": w["probes"], "lanczos_steps": args.t,
            "residual_check": True, "l2": "flushed between steps (256 MiB write, outside step events)"}


def workload(args):
    from paper_2405_03474_gb300 import inputs
    w = dict(inputs.WORKLOADS[WORKLOAD])
    w["n"] = args.n
    return w


# ------------------------------------------------------------------ CPU side
_SH = {}


def _attach(names):
    """Pool initializer: map the parent's shared X and V blocks (no copies)."""
    import numpy as np
    from multiprocessing import shared_memory
    for key, (name, shape) in names.items():
        shm = shared_memory.SharedMemory(name=name)
        _SH[key] = (shm, np.ndarray(shape, dtype=np.float64, buffer=shm.buf))


def _oracle_rows(job):
    """Worker: the oracle's matrix-free rows of (K + nu I) V and the seconds they take."""
    rows, ncols, ell, nu = job
    import numpy as np
    from oracle import kernels
    X = _SH["X"][1]
    V = _SH["V%d" % ncols][1]
    t0 = time.perf_counter()
    out = kernels.kz_rows(X, V, np.asarray(rows), kernels.MATERN52, ell, 1.0, nu)
    return time.perf_counter() - t0, out


class OraclePool:
    """Process pool (spawn, one process per host core, one BLAS thread each)
    sharing the workload's points and V blocks through shared memory."""

    def __init__(self, w):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        import numpy as np
        from paper_2405_03474_gb300 import inputs
        self.w = w
        self.cores = os.cpu_count() or 1
        n, d = w["n"], w["d"]
        arrays = {"X": inputs.points(n, d, w["dist"], seed=inputs.SEED_POINTS)}
        self.cols = sorted({w["probes"], w["probes"] * w["order"], w["rank"]})
        for c in self.cols:
            arrays["V%d" % c] = inputs.gaussian(n, c, seed=5)
        self.shm, names = [], {}
        for key, arr in arrays.items():
            shm = shared_memory.SharedMemory(create=True, size=arr.nbytes)
            np.ndarray(arr.shape, dtype=np.float64, buffer=shm.buf)[...] = arr
            self.shm.append(shm)
            names[key] = (shm.name, arr.shape)
        del arrays
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_attach, initargs=(names,))
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

    def estimate_seconds(self, t_steps, rows_per_core=None):
        """Seconds the CPU oracle needs for one estimate of the workload,
        extrapolated from its matrix-free K V on a sample of rows (all cores in
        parallel): (q + 2) sketch products with `rank` columns, t CG products with
        `probes` columns and one residual product with probes * order columns."""
        w = self.w
        n = w["n"]
        per_pass = {}
        rows_per_core = rows_per_core or ROWS_PER_CORE
        sample_rows = rows_per_core * self.cores
        import numpy as np
        stride = max(1, n // sample_rows)  # rows spread over the whole point set
        for ncols in self.cols:
            jobs = [([(c * rows_per_core + k) * stride for k in range(rows_per_core)], ncols, w["lengthscale"],
                     w["noise"]) for c in range(self.cores)]
            got = self.pool.map(_oracle_rows, jobs)
            per_pass[ncols] = max(g[0] for g in got) * n / sample_rows
            if ncols == w["probes"]:
                # the sampled rows double as the FP64 reference of the product's error
                self.rows = np.concatenate([j[0] for j in jobs])
                self.values = np.concatenate([g[1] for g in got])
        total = ((w["power_iters"] + 2) * per_pass[w["rank"]] + t_steps * per_pass[w["probes"]]
                 + per_pass[w["probes"] * w["order"]])
        sample = ("oracle kernels.kz_rows on %d of %d rows for V with %s columns, %d processes x 1 "
                  "thread; extrapolated to (q+2)=%d sketch + t=%d CG + 1 residual K V passes "
                  "(the oracle's n-by-r and scalar work is not counted)"
                  % (sample_rows, n, "/".join(str(c) for c in self.cols), self.cores,
                     w["power_iters"] + 2, t_steps))
        return total, sample

    def close(self):
        self.pool.terminate()
        for shm in self.shm:
            shm.close()
            shm.unlink()


# ------------------------------------------------------------------ GPU side
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        mhz, mx, reasons, power = [], None, set(), []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                  "sw_power_cap"), f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        busy = [m for m in mhz if mx and m > 0.5 * mx] or mhz
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz),
                "power_w_max": max(power) if power else None}


def run_ours(args, rank, world, local_rank, pool):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2405_03474_gb300 import _lib, api, inputs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    lib = _lib.load()
    w = workload(args)
    n, d = w["n"], w["d"]
    kern = api.Kernel(w["kind"], w["lengthscale"], w["variance"], w["noise"])
    X_host = torch.as_tensor(inputs.points(n, d, w["dist"], seed=inputs.SEED_POINTS)).pin_memory()
    X = X_host.to(dev)
    opts = dict(order=w["order"], num_probes=w["probes"], probes_per_block=w["probes"],
                fixed_iters=args.t, max_iters=args.t, precision=args.precision, residual_check=True,
                seed=rank_probe_seed(rank))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step(Xd, mid=None):
        P = api.Precond.build(Xd, kern, w["rank"], power_iters=w["power_iters"],
                              seed=inputs.SEED_SKETCH, precision=args.sketch_precision)
        if mid is not None:
            mid.record(torch.cuda.current_stream())  # preconditioner built
        res = api.logdet_estimate(Xd, kern, precond=P, **opts)
        P.free()
        return res

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        res = step(X)
    torch.cuda.synchronize()

    # timed region: K steps, L2 flushed between steps (outside the step events)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = Clocks(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = lib.ld_launch_count()
    lib.ld_profile_begin()
    results = []
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        results.append(step(X, mids[k]))
        ev[k][1].record(stream)
    import ctypes
    kz_ms, kz_n, kz_pairs, kz_flops = (ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(),
                                      ctypes.c_double())
    lib.ld_profile_end(ctypes.byref(kz_ms), ctypes.byref(kz_n), ctypes.byref(kz_pairs), ctypes.byref(kz_flops))
    per_kernel = {}
    for kid, kname_ in ((1, "kz_sym_kernel"), (4, "kz_wide_kernel"), (0, "kz_tc_kernel")):
        m_, n_, p_, f_ = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        lib.ld_profile_kernel(kid, ctypes.byref(m_), ctypes.byref(n_), ctypes.byref(p_), ctypes.byref(f_))
        per_kernel[kname_] = (m_.value, n_.value, p_.value, f_.value)
    torch.cuda.synchronize()
    barrier()
    launches = lib.ld_launch_count() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    build_ms = [ev[k][0].elapsed_time(mids[k]) for k in range(args.steps)]
    total_ms = sum(step_ms)
    total_ms_max = max_over_ranks(total_ms, world, dev)
    value = job_value(world, args.steps, total_ms_max)

    # end to end through the public API: host points in, host result out
    e2e = None
    if not args.no_e2e:
        e2e_ms = []
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            Xd = X_host.to(dev, non_blocking=True)
            r = step(Xd)  # returns host scalars and the host per-probe array
            b.record(stream)
            torch.cuda.synchronize()
            e2e_ms.append(a.elapsed_time(b))
        e2e = {"value": job_value(world, args.steps, max_over_ranks(sum(e2e_ms), world, dev)), "unit": UNIT,
               "h2d_bytes_per_step": int(X_host.numel() * X_host.element_size()),
               "d2h_bytes_per_step": int(8 * (w["probes"] + 16))}

    if rank != 0:
        return None

    # The same estimate in other precisions, once each after the timed region: one
    # preconditioner (built as in the timed step) and the same device-drawn probes, so
    # the estimates differ only by the arithmetic of the products and CG; time by CUDA
    # events around each call, relative difference from the timed precision's estimate.
    estimate_compare = None
    precs = [p_ for p_ in args.estimate_compare.split(",") if p_]
    if precs:
        Pc = api.Precond.build(X, kern, w["rank"], power_iters=w["power_iters"], seed=inputs.SEED_SKETCH,
                               precision=args.sketch_precision)
        handles = {"f32": Pc}

        def timed_estimate(prec):
            if prec == "fp64" and "f64" not in handles:
                A_, D_, _ = Pc.export()
                handles["f64"] = api.Precond.import_(A_, D_, "fp64")
                del A_, D_
            Ph = handles["f64" if prec == "fp64" else "f32"]
            torch.cuda.synchronize()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            r_ = api.logdet_estimate(X, kern, precond=Ph, **dict(opts, precision=prec))
            b_.record(stream)
            torch.cuda.synchronize()
            return a_.elapsed_time(b_), r_

        ms_ref, r_ref = timed_estimate(args.precision)
        estimate_compare = {"reference_precision": args.precision, "ms": ms_ref, "logdet": r_ref["logdet"],
                            "std_err": r_ref["std_err"], "max_resid": r_ref["max_resid"][:w["order"]],
                            "note": "same preconditioner (built once, sketch %s) and probes; ms excludes the "
                                    "preconditioner build" % args.sketch_precision}
        for prec in precs:
            ms_p, r_p = timed_estimate(prec)
            estimate_compare[prec] = {"ms": ms_p, "logdet": r_p["logdet"], "logdet_P": r_p["logdet_P"],
                                      "rel_diff": abs(r_p["logdet"] - r_ref["logdet"]) / abs(r_p["logdet"]),
                                      "max_resid": r_p["max_resid"][:w["order"]],
                                      "speedup_of_%s" % args.precision: ms_p / ms_ref}
        for h in handles.values():
            h.free()

    grad_side = None if args.no_grad_side else gradient_side(stream)

    kname = "matern52" if w["kind"] == inputs.MATERN52 else "rbf"
    peak = pair_peak_gps(kname, d)
    tc_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("bf16_tflops") \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else None

    def roof(name):
        """ALU roofline of one kernel over the timed region: distinct kernel evaluations
        per launch over the launch's average CUDA-event time."""
        ms, nl, pairs, flops = per_kernel[name]
        if nl == 0:
            return None
        avg = ms / nl
        ach = pairs / nl / (avg / 1e3) / 1e9
        out = {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "Gpair/s",
               "frac": ach / peak, "traffic": None, "launches": nl, "avg_launch_ms": avg,
               "share_of_step": ms / total_ms, "tensor_tflops": flops / (ms / 1e3) / 1e12,
               "peak_note": "ALU roofline of the pair evaluation derived from measured GB300 pipe rates"}
        if tc_peak:
            out["tensor_frac_of_measured_bf16"] = out["tensor_tflops"] / tc_peak
        return out

    sym_roof = roof("kz_sym_kernel")
    if sym_roof:
        sym_roof["traffic"] = measured_traffic(KZ_SYM_TRAFFIC)
        sym_roof["traffic_note"] = ("DRAM bytes per launch from one ncu capture (n=2^20, 16 columns); the "
                                    "algorithmic DRAM bytes of a matrix-free launch are only its inputs and "
                                    "output (X tiles, V image, W in tile order: ~0.2 GB); the rest is L2 "
                                    "spill of the V image and W at this n")
    roofs = [r for r in (sym_roof, roof("kz_wide_kernel"), roof("kz_tc_kernel")) if r]
    roofs.sort(key=lambda r: -r["share_of_step"])
    dominant, others = (roofs[0] if roofs else None), roofs[1:]
    res = results[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16x3", "data": "synthetic",
        "config": dict(config_of(args, w), kz_precision=args.precision, sketch_precision=args.sketch_precision,
                       parallelism="independent estimate per GPU"),
        "probe_matvecs_per_s": world * args.steps * (w["probes"] * args.t + w["probes"] * w["order"])
                               / (total_ms_max / 1e3),
        "sketch_matvecs_per_s": world * args.steps * (w["power_iters"] + 2) * w["rank"] / (total_ms_max / 1e3),
        "precond_build_ms": statistics.mean(build_ms),
        "estimates_per_s_precond_amortised": 1e3 / statistics.mean(
            [s_ - b_ for s_, b_ in zip(step_ms, build_ms)]) * world,
        "estimate": {"logdet": res["logdet"], "logdet_P": res["logdet_P"], "std_err": res["std_err"],
                     "iters": res["iters"], "max_resid": res["max_resid"][:w["order"]]},
        "roofline": dominant,
        "roofline_other_kernels": others,
        "kernel_products": {"launches": kz_n.value, "device_ms": kz_ms.value, "share_of_step": kz_ms.value / total_ms,
                            "product_pairs_per_s": sum(v[1] for v in per_kernel.values())
                            * float(n) * n / (kz_ms.value / 1e3) if kz_ms.value else None},
        "clocks": clk,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "estimate_precision_compare": estimate_compare,
        "gradient_side": grad_side,
    }
    if pool is not None:
        sec, sample = pool.estimate_seconds(args.t)
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                                "sample": sample}
        # error of the timed product (hi/lo fp16 tensor cores, 16 columns) on the rows the
        # baseline computed in FP64, same V
        V = torch.as_tensor(inputs.gaussian(n, w["probes"], seed=5), dtype=torch.float32).to(dev)
        Wg = api.ld_kz(X, V, kern, args.precision)[torch.as_tensor(pool.rows, device=dev)].double().cpu().numpy()
        line["kz_rel_err_vs_fp64_oracle"] = {
            "value": float(np.linalg.norm(Wg - pool.values) / np.linalg.norm(pool.values)),
            "rows": int(len(pool.rows)), "columns": w["probes"], "precision": args.precision}
        # the same product in every precision (one launch each, after the timed region):
        # time and error on the same FP64 rows, i.e. the speedup at a stated accuracy
        if not args.no_precision_compare:
            cmp = {}
            idx = torch.as_tensor(pool.rows, device=dev)
            for prec in ("fp32", "f16x3_tc", "f16_tc", "bf16_tc"):
                api.ld_kz(X, V, kern, prec)  # warm (workspace, first-launch costs)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                Wp = api.ld_kz(X, V, kern, prec)
                b.record(stream)
                torch.cuda.synchronize()
                Wr = Wp[idx].double().cpu().numpy()
                cmp[prec] = {"ms": a.elapsed_time(b),
                             "rel_err": float(np.linalg.norm(Wr - pool.values) / np.linalg.norm(pool.values))}
            for prec in cmp:
                cmp[prec]["speedup_vs_fp32"] = cmp["fp32"]["ms"] / cmp[prec]["ms"]
            line["kz_precision_compare"] = {"columns": w["probes"], "n": n, **cmp}
    return line


def gradient_side(stream):
    """The hand-written adjoint on the gradient workload's points (n = 2^17 uniform in
    [0,1]^2, RBF, 16 probes, rank-128 preconditioner), once in hi/lo fp16 on the tensor
    cores and once in FP32 SIMT with the same preconditioner and probes, at the
    hyperparameters (0.2, 1, 0.1) where the hi/lo fp16 operator is well inside positive
    definiteness; time by CUDA events (the preconditioner build excluded) and the
    relative difference of the two gradients."""
    import numpy as np
    import torch
    from paper_2405_03474_gb300 import api, inputs
    w = inputs.WORKLOADS["rbf_grad_n131072_d2"]
    th = (0.2, 1.0, 0.1)
    n, d, s_ = w["n"], w["d"], 16
    X = torch.as_tensor(inputs.points(n, d, w["dist"], seed=inputs.SEED_POINTS)).cuda()
    kern = api.Kernel(w["kind"], *th)
    P = api.Precond.build(X, kern, w["rank"], power_iters=w["power_iters"], seed=inputs.SEED_SKETCH,
                          precision="f16_tc")
    Z = torch.as_tensor(inputs.rademacher(n, s_, seed=inputs.SEED_PROBES)).cuda()
    out = {"workload": "rbf_grad_n131072_d2", "theta": th, "probes": s_, "rank": w["rank"], "rel_tol": 1e-6}
    for prec in ("f16x3_tc", "fp32"):
        api.logdet_grad(X, kern, precond=P, probes=Z, order=3, num_probes=s_, precision=prec, rel_tol=1e-6,
                        max_iters=3000)  # warm
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = api.logdet_grad(X, kern, precond=P, probes=Z, order=3, num_probes=s_, precision=prec, rel_tol=1e-6,
                            max_iters=3000)
        b.record(stream)
        torch.cuda.synchronize()
        out[prec] = {"ms": a.elapsed_time(b), "grad": [float(g) for g in r["grad"]], "iters": r["iters"],
                     "logdet": r["logdet"]}
    g16, g32 = np.array(out["f16x3_tc"]["grad"]), np.array(out["fp32"]["grad"])
    out["rel_diff"] = [float(v) for v in np.abs(g16 - g32) / np.abs(g32)]
    out["speedup_of_f16x3_tc"] = out["fp32"]["ms"] / out["f16x3_tc"]["ms"]
    P.free()
    return out


def run_reference(args, pool):
    """The oracle timed on the host cores: per step, the same row sample (ROWS_PER_CORE
    rows per core of every product width) as our arm's cpu_baseline leg, extrapolated
    to one estimate; the warm-up steps are sampled and discarded."""
    w = workload(args)
    cores = pool.cores
    vals = []
    sample = ""
    for k in range(args.warmup + args.steps):
        sec, sample = pool.estimate_seconds(args.t, rows_per_core=ROWS_PER_CORE)
        if k >= args.warmup:
            vals.append(1.0 / sec)
    value = statistics.mean(vals)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": dict(config_of(args, w), kz_precision="fp64 (oracle)", sketch_precision="fp64 (oracle)",
                           parallelism="host cores (process pool)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_kz_only(args):
    """Small case for ncu: the kernel product of the workload on C columns."""
    import torch
    from paper_2405_03474_gb300 import api, inputs
    w = workload(args)
    X = torch.as_tensor(inputs.points(w["n"], w["d"], w["dist"], seed=inputs.SEED_POINTS)).cuda()
    V = torch.as_tensor(inputs.gaussian(w["n"], args.kz_only, seed=7), dtype=torch.float32).cuda()
    kern = api.Kernel(w["kind"], w["lengthscale"], w["variance"], w["noise"])
    for _ in range(3):
        W = api.ld_kz(X, V, kern, args.precision)
    torch.cuda.synchronize()
    print(json.dumps({"kz_only": True, "n": w["n"], "c": args.kz_only, "precision": args.precision,
                      "checksum": float(W.double().abs().sum())}))
    return 0


def run_dense_only(args):
    """Small case for ncu: the stored-M tensor-core product, N points of the stored-dense workload."""
    import torch
    from paper_2405_03474_gb300 import api, inputs
    w = inputs.WORKLOADS["rbf_n65536_d3"]
    n = args.dense_only
    X = torch.as_tensor(inputs.points(n, w["d"], w["dist"], seed=inputs.SEED_POINTS)).cuda()
    M = api.ld_dense_materialize(X, api.Kernel(w["kind"], w["lengthscale"], w["variance"], w["noise"]), "fp32")
    V = torch.as_tensor(inputs.gaussian(n, 64, seed=2), dtype=torch.float32).cuda()
    for _ in range(3):
        W = api.ld_dense_kz(M, V, "f16x3_tc")
    torch.cuda.synchronize()
    print(json.dumps({"dense_only": True, "n": n, "c": 64, "checksum": float(W.double().abs().sum())}))
    return 0


def run_cg_only(args):
    """Small case for ncu: one estimate of the workload with a rank-64 preconditioner and t = 2."""
    import torch
    from paper_2405_03474_gb300 import api, inputs
    w = workload(args)
    X = torch.as_tensor(inputs.points(w["n"], w["d"], w["dist"], seed=inputs.SEED_POINTS)).cuda()
    kern = api.Kernel(w["kind"], w["lengthscale"], w["variance"], w["noise"])
    P = api.Precond.build(X, kern, 64, power_iters=1, seed=inputs.SEED_SKETCH, precision=args.sketch_precision)
    r = api.logdet_estimate(X, kern, precond=P, order=w["order"], num_probes=w["probes"], fixed_iters=2,
                            max_iters=2, precision=args.precision, residual_check=True)
    print(json.dumps({"cg_only": True, "n": w["n"], "logdet": r["logdet"]}))
    return 0


def main():
    args = parse()
    if args.kz_only:
        return run_kz_only(args)
    if args.dense_only:
        return run_dense_only(args)
    if args.cg_only:
        return run_cg_only(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        pool = OraclePool(workload(args))
        try:
            line = run_reference(args, pool)
        finally:
            pool.close()
        print(json.dumps(line))
        return 0
    # the oracle's process pool is started (spawn) before any GPU call
    pool = None
    if rank == 0 and not args.no_cpu:
        pool = OraclePool(workload(args))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        line = run_ours(args, rank, world, local_rank, pool)
    finally:
        if pool is not None:
            pool.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
