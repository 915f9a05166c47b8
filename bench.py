"""Benchmark: seconds to M Karhunen-Loeve eigenpairs on one GB300.

Workload (default): unit cube, p = 2, 16 x 16 x 16 elements (N = 5832 trial
dofs), separable exponential kernel exp(-sum_d |x_d - x'_d| / L), L = 1,
sigma = 1, M = 20 eigenpairs, eigensolver block k = 8. One step is one
complete solve by the IBQ-Galerkin method (N~ = 35937 interpolation points,
1.29e9 kernel pairs per operator application) followed by one by the
collocation method (110592 quadrature points, 6.45e8 pairs per
application), both with the mixed-precision pairwise path (FP32 kernel tiles,
split BF16 tcgen05 products, FP64 Rayleigh-Ritz refinement).

The line also reports the plain FP64 GPU solves of the same step, the
relative eigenvalue error of every mixed-precision eigenvalue against them,
the roofline of the dominant kernel, end-to-end time through the C ABI with
host buffers, and the FP64 CPU oracle on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "cube_p2_e16_expsep"
# (special-function ops, FP32 ops) per kernel evaluation Gamma(x, x') with
# pre-scaled coordinates: 3 differences + the argument (2 adds of |d| for the
# separable exponential; 1 mul + 2 fma for the squared distance) + the
# Matern factor (1 fma, 1 mul); ex2, and sqrt for the Euclidean distance
ALU_OPS_PER_PAIR = {"gauss": (1, 6), "exp_sep": (1, 5), "exp": (2, 6), "matern32": (2, 8), "const": (1, 1)}
METHODS = ("galerkin", "collocation")
MIXED = "bf16"
# SMs each solve's pairwise product leaves free in the concurrent step
# (kl_set_shared_sms; measured on GB300: 8 of 152 gave the shortest step)
SHARED_SMS = 8


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default=MIXED, choices=["bf16", "tf32", "fp32"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU comparison solves")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--profile-step", action="store_true",
                    help="run exactly one untimed step (for ncu launch lists); prints nothing")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="workload of kl_inputs.WORKLOADS (default: the 16^3 cube, the benchmark's configuration)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving (continuous batching) leg")
    ap.add_argument("--autotune", action="store_true",
                    help="choose each method's block size with kl_autotune (complete solves for k = 8, 16, 32, "
                         "before the timed region) instead of the workload's k")
    ap.add_argument("--serve-requests", type=int, default=64,
                    help="requests of the seeded serving stream replayed by the serving leg")
    ap.add_argument("--serve-max-elems", type=int, default=8,
                    help="per-axis element cap of the serving stream sample")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the annulus workloads (quarter annular cylinder, p = 3 Gaussian and p = 2 exponential)")
    ap.add_argument("--configs-fp64", action="store_true",
                    help="also solve the 64x32x16 annulus workload in FP64 (minutes of FP64 GPU time)")
    ap.add_argument("--accuracy", action="store_true",
                    help="accuracy-versus-time study instead of the benchmark: every method on a sequence of cube "
                         "meshes against the standard Gauss-Legendre Galerkin solution on the finest one")
    ap.add_argument("--accuracy-elems", default="4,8,12,16", help="per-axis element counts of the study")
    ap.add_argument("--accuracy-kernel", default="exp_sep", choices=["gauss", "exp_sep", "exp", "matern32"])
    ap.add_argument("--accuracy-study", default="cube", choices=["cube", "paper"],
                    help="cube: h-refined unit cubes; paper: the half-cylinder cases of Tables 1-2 (Sec. 4)")
    return ap.parse_args()


def max_over_ranks(x, dist, device):
    """Replicas: every rank solves its own instance; the job's step time is
    the slowest rank's (all ranks see it)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _recorded_traffic(kernel_class):
    """DRAM bytes per launch of the pairwise kernel class from the committed
    ncu summary, if it covers that class and the kernel source is unchanged
    since it was taken (else None)."""
    import hashlib
    try:
        rec = {}
        for line in open(os.path.join(ROOT, "profiles", "pair_tc_kernel_traffic.txt")):
            if ":" in line:
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
        if rec.get("kernel_class") != kernel_class:
            return None
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
        if hashlib.sha1(src).hexdigest() != rec["source_sha1"]:
            return None
        return int(rec["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def _sampling_leg(kl, handles, streams, lam, Vd, N, M, args, fp64_fma, ns=1024, reps=5):
    """Realisations of the truncated expansion (Sec. 2) from each method's
    eigenpairs: kl_sample at the tensor Gauss grid, ns samples per call, timed
    with CUDA events on the handle's stream. On GB300 the FP64 FMAs bound it,
    not HBM: the coefficient GEMM (N M ns) and the three banded passes of the
    sum factorisation (p + 1 trial functions per Gauss point and direction,
    direction 1 first: Ne1 N2 N3, Ne1 Ne2 N3 and Ne1 Ne2 Ne3 outputs per
    sample). HBM figures beside it: the inputs and the output (V: N x M,
    xi: M x ns, the samples: Q x ns, FP64) as algorithmic bytes."""
    import numpy as np
    import torch

    peaks, src = _peaks()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2101)
    out = {}
    for m, h in handles.items():
        Q = kl.kl_sample_size(h)
        xi = torch.randn((ns, M), dtype=torch.float64, device="cuda", generator=gen)  # column-major M x ns
        res = torch.empty((ns, Q), dtype=torch.float64, device="cuda")
        st = streams[m]
        torch.cuda.synchronize()
        for _ in range(2):
            kl.kl_sample(h, M, lam[m], Vd[m], N, xi, M, ns, res, Q)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            kl.kl_sample(h, M, lam[m], Vd[m], N, xi, M, ns, res, Q)
        e1.record(st)
        e1.synchronize()
        t = e0.elapsed_time(e1) / reps * 1e-3
        alg = 8 * (N * M + M * ns + Q * ns)
        p = args["p"]
        n1 = [e + p for e in args["elems"]]           # trial functions per direction (C^{p-1})
        ne = [(p + 1) * e for e in args["elems"]]     # Gauss points per direction
        fma = ns * (N * M + (p + 1) * (ne[0] * n1[1] * n1[2] + ne[0] * ne[1] * n1[2] + ne[0] * ne[1] * ne[2]))
        out[m] = {"ns": ns, "Q": Q, "ms": t * 1e3, "samples_per_s": ns / t,
                  "bound": "fp64", "fma_per_call": fma, "achieved_tfma": fma / t / 1e12,
                  "peak_tfma": fp64_fma / 1e12, "frac": fma / t / fp64_fma,
                  "bytes_per_call": alg, "achieved_gbs": alg / t / 1e9, "peak_gbs": peaks["hbm_gbs"],
                  "peak_gbs_source": src, "frac_hbm": alg / t / 1e9 / peaks["hbm_gbs"],
                  "finite": bool(torch.isfinite(res).all().item())}
        del res, xi
    return out


def _serve_leg(a, kl, stream):
    """Replays a bounded sample of the seeded serving stream (Poisson
    arrivals) through kl_serve_*, then the same requests one at a time."""
    import numpy as np
    import torch
    from kl_inputs import serving_requests

    reqs = serving_requests(a.serve_requests, seed=2101, max_elems=a.serve_max_elems, mean_interarrival_s=0.02)

    def prm(r, precision):
        return kl.params(geometry=r["geometry"], degree=r["p"], elems=r["elems"], kernel=r["kernel"],
                         sigma=r["sigma"], L=r["L"], method=r["method"], precision=precision, block_k=8,
                         seed=5 + r["id"])

    # untimed warm-up of the batched path (module load, first launches)
    s = kl.kl_serve_open(0, a.serve_slots, 0)
    warm = [np.zeros(reqs[i]["M"]) for i in range(min(2, len(reqs)))]
    for i, buf in enumerate(warm):
        kl.kl_serve_submit(s, prm(reqs[i], a.precision), reqs[i]["M"], 0.0, i, buf)
    got = 0
    while got < len(warm):
        got += len(kl.kl_serve_poll(s, 16, 500))
    kl.kl_serve_close(s)

    s = kl.kl_serve_open(0, a.serve_slots, 0)
    bufs = [np.zeros(r["M"]) for r in reqs]
    results = {}
    t0 = time.perf_counter()
    for r, buf in zip(reqs, bufs):
        while time.perf_counter() - t0 < r["t"]:
            for x in kl.kl_serve_poll(s, 64, 0):
                results[x["request_id"]] = (x, time.perf_counter() - t0)
            time.sleep(0.0005)
        kl.kl_serve_submit(s, prm(r, a.precision), r["M"], 0.0, r["id"], buf)
    while len(results) < len(reqs):
        for x in kl.kl_serve_poll(s, 64, 200):
            results[x["request_id"]] = (x, time.perf_counter() - t0)
    wall = max(t for _, t in results.values())
    stats = kl.kl_serve_get_stats(s)
    kl.kl_serve_close(s)
    lat = [x["latency_ms"] for x, _ in results.values()]
    pairs = sum(r["M"] for r in reqs)
    bad_status = sorted(x["status"] for x, _ in results.values() if x["status"] not in (0, 1))
    bad = len(bad_status)
    failed_requests = [dict({k: reqs[int(x["request_id"])][k] for k in ("id", "geometry", "p", "elems", "kernel", "L",
                                                                        "M", "method")},
                            status=x["status"], applies=x["applies"], restarts=x["restarts"],
                            max_resid=x["max_resid"])
                       for x, _ in results.values() if x["status"] not in (0, 1)]

    # the same requests one at a time (no batching, no overlap)
    def one(r, precision):
        h = kl.kl_create(prm(r, precision), stream)
        lam = np.zeros(r["M"])
        torch.cuda.synchronize()
        t = time.perf_counter()
        kl.kl_eigs(h, r["M"], 0.0, lam, None, 0, 0)
        dt = time.perf_counter() - t
        kl.kl_destroy(h)
        return dt, lam

    seq = [one(r, a.precision) for r in reqs]
    seq_s = sum(d for d, _ in seq)
    # agreement of the served eigenvalues with the one-at-a-time solves
    agree = max(float(np.max(np.abs(bufs[i] - seq[i][1]) / np.maximum(np.abs(seq[i][1]), 1e-6 * abs(seq[i][1][0]))))
                for i in range(len(reqs)))
    nfp = min(4, len(reqs))
    fp64 = [one(reqs[i], "fp64")[0] for i in range(nfp)]
    return {
        "workload": "seeded Poisson stream of K-L requests (cube/annulus, p 2-4, Gauss/exp/Matern-3/2, "
                    "L log-uniform 0.1-2, M 10-100, Galerkin/collocation)",
        "sample": f"first {len(reqs)} requests, per-axis elements <= {a.serve_max_elems}, mean inter-arrival 20 ms",
        "precision": a.precision, "slots": a.serve_slots, "requests": len(reqs), "failed": bad,
        "failed_status": bad_status, "failed_requests": failed_requests,
        "wall_s": wall, "eigenpairs_per_s": pairs / wall,
        "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
        "queue_ms_p50": float(np.percentile([x["queue_ms"] for x, _ in results.values()], 50)),
        "batches": stats["batches"], "batched_products": stats["batched_products"], "max_batch": stats["max_batch"],
        "max_concurrent": stats["max_concurrent"],
        "one_at_a_time_s": seq_s, "throughput_vs_one_at_a_time": seq_s / wall,
        "max_lam_rel_diff_vs_one_at_a_time": agree,
        "fp64_one_at_a_time_s_first": {"requests": nfp, "fp64_s": sum(fp64),
                                       "mixed_s": sum(seq[i][0] for i in range(nfp))},
    }


# --------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and --impl reference): the dense FP64 oracle,
# timed as it stands on a bounded sample of the workload: the same cube
# problem (p = 2, separable exponential kernel, M = 20, both methods) on a
# coarser mesh. At the full 16^3 mesh the oracle cannot run within a
# benchmark: its Galerkin form factors dense N~ x N~ matrices (N~ = 35937:
# 10 GB each, about 2.5e14 flops of dense solves) and its collocation form
# multiplies a dense 5832 x 110592 kernel matrix. So every value below is a
# measured time of the sample, never an extrapolation; the GPU's time on the
# same sample problem is measured beside it.
# --------------------------------------------------------------------------
METRIC = "s to M K-L eigenpairs (Galerkin + collocation solve)"
CPU_SAMPLE_ELEMS = 8


def _oracle_sample(n=CPU_SAMPLE_ELEMS):
    """Seconds of one dense-oracle step (both methods) on the n^3 sample."""
    from kl_inputs import WORKLOADS, problem_args
    from oracle import collocation, galerkin
    from oracle.problem import Problem

    w = WORKLOADS[WORKLOAD]
    args = problem_args(w)
    per = {}
    for method in METHODS:
        prob = Problem(args["geometry"], args["p"], (n, n, n), args["kernel"], args["sigma"], args["L"])
        mod = galerkin if method == "galerkin" else collocation
        t0 = time.perf_counter()
        mod.solve(prob, w["M"])
        per[method] = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return sum(per.values()), per, cores


def _sample_text(n, per):
    return (f"dense FP64 oracle (scipy eigh / QZ on assembled matrices) on the {n}^3-element mesh of the "
            f"{WORKLOAD} problem (p = 2, separable exponential, L = 1, M = 20, both methods): measured "
            f"{per['galerkin']:.2f} s Galerkin + {per['collocation']:.2f} s collocation; the full "
            f"16^3 step does not fit a benchmark run (dense N~ x N~ factorisations, N~ = 35937)")


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    n = 7 if a.steps > 8 else CPU_SAMPLE_ELEMS  # bounded: the whole run stays within minutes
    for _ in range(min(a.warmup, 1)):
        _oracle_sample(n)  # warm-up (imports, BLAS thread pools)
    vals, pers = [], []
    for _ in range(a.steps):
        v, per, cores = _oracle_sample(n)
        vals.append(v)
        pers.append(per)
    v = float(np.median(vals))
    per = {m: float(np.median([p[m] for p in pers])) for m in METHODS}
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": v, "unit": "s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "M": 20, "k": 8, "methods": list(METHODS),
                   "step": f"bounded sample: the {n}^3 mesh of the workload's problem, both methods"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle", "sample": _sample_text(n, per)},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() in ("active", "1"):
                    reasons.add(name)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _lam_err(lam, ref):
    import numpy as np
    return np.abs(lam - ref) / np.maximum(np.abs(ref), 1e-6 * abs(ref[0]))


def _timed_solve(kl, torch, stream, h, M, tol, lam, info):
    """One kl_eigs on the handle's stream between CUDA events (seconds)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc = kl.kl_eigs(h, M, tol, lam, None, 0, 0, None, info)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3, rc


def _pair_roof(kernel, peaks):
    """ALU roof (pairs/s) of one kernel evaluation (see the roofline block)."""
    fp32_fma, ex2, _ = peaks
    mufu, fp32 = ALU_OPS_PER_PAIR[kernel]
    return min(ex2 / mufu, fp32_fma / fp32)


# Block sizes of the annulus workloads: kl_autotune's choice on GB300 for the
# exponential one (complete solves for k = 8, 16, 32: Galerkin 2.22 / 1.56 /
# 1.52 s, collocation 1.25 / 0.93 / 1.08 s), the workload's k otherwise.
CONFIG_WORKLOADS = (("annulus_p3_e32x32x16_gauss", {"galerkin": 16, "collocation": 16}),
                    ("annulus_p2_e64x32x16_exp", {"galerkin": 32, "collocation": 16}))


def _configs_leg(a, kl, stream, peaks):
    """The quarter-annulus workloads: per method one untimed and one timed
    mixed-precision solve (CUDA events), the pairwise kernel's rate during
    the timed solve against its ALU roof, and FP64 solves of the same problem
    stopped at the mixed solve's tolerance (the smaller workload by default;
    both with --configs-fp64) with the eigenvalue errors of the mixed pairs
    against them."""
    import numpy as np
    import torch
    from kl_inputs import WORKLOADS, problem_args

    out = {}
    for name, ks in CONFIG_WORKLOADS:
        w = WORKLOADS[name]
        args = problem_args(w)
        M = w["M"]
        res = {}
        for m in METHODS:
            def mk(precision):
                p = kl.params(geometry=args["geometry"], degree=args["p"], elems=args["elems"], kernel=args["kernel"],
                              sigma=args["sigma"], L=args["L"], geo=args.get("geo", (1.0, 2.0, 1.0)), method=m,
                              precision=precision, block_k=ks[m], seed=2101)
                return kl.kl_create(p, stream)
            h = mk(a.precision)
            dims = kl.kl_dims(h)
            lam = np.zeros(M)
            info = kl.kl_solve_info()
            _timed_solve(kl, torch, stream, h, M, 0.0, lam, info)  # untimed: graphs, workspaces
            kl.kl_profile_enable(h, True)
            t, rc = _timed_solve(kl, torch, stream, h, M, 0.0, lam, info)
            prof = kl.kl_profile_read(h)
            kl.kl_profile_enable(h, False)
            kl.kl_destroy(h)
            # the symmetric Galerkin class counts each symmetric pair once (its
            # kernel evaluates each once); the dense classes every pair
            pair_key = next((key for key in ("pair_tc_%s_sym" % a.precision, "pair_tc_" + a.precision, "pair_f32")
                             if key in prof), None)
            pair = prof.get(pair_key) if pair_key else None
            r = dict(N=dims[0], pairwise_sources=dims[1], pairwise_targets=dims[2], k=ks[m], status=rc, s=t,
                     applies=info.applies, max_resid=info.max_resid)
            if pair:
                rate = pair["units"] / (pair["ms"] * 1e-3)
                r["pairwise"] = dict(kernel_class=pair_key, launches=pair["launches"], ms=pair["ms"],
                                     gpairs_per_s=rate / 1e9,
                                     frac_alu_roof=rate / _pair_roof(args["kernel"], peaks),
                                     share_of_solve=pair["ms"] * 1e-3 / t)
            if name == CONFIG_WORKLOADS[0][0] or a.configs_fp64:
                h64 = mk("fp64")
                lam64 = np.zeros(M)
                info64 = kl.kl_solve_info()
                t64, rc64 = _timed_solve(kl, torch, stream, h64, M, 1e-6, lam64, info64)
                kl.kl_destroy(h64)
                err = _lam_err(lam, lam64)
                r["fp64_matched_tol"] = dict(tol=1e-6, s=t64, status=rc64, applies=info64.applies,
                                             speedup=t64 / t, max_lam_rel_err=float(err.max()))
            res[m] = r
        out[name] = dict(M=M, methods=res)
    return out


def run_gpu(a):
    import numpy as np
    import torch

    import paper_2101_00629_gb300 as kl
    from kl_inputs import WORKLOADS, problem_args

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    w = WORKLOADS[a.workload]
    args = problem_args(w)
    geo = args.get("geo", (1.0, 2.0, 1.0))  # geometry parameters (annulus radii and height by default)
    M, k = w["M"], w["k"]
    ks = {m: k for m in METHODS}
    tuned = {}
    if a.autotune:
        for m in METHODS:
            pt = kl.params(geometry=args["geometry"], degree=args["p"], elems=args["elems"], kernel=args["kernel"],
                           sigma=args["sigma"], L=args["L"], geo=geo, method=m, precision=a.precision, block_k=8,
                           seed=2101 + 7919 * rank)
            best, secs = kl.kl_autotune(pt, M, 0.0, stream)
            ks[m] = best
            tuned[m] = {"k": best, "solve_s": {str(c): (round(t, 4) if t >= 0 else None) for c, t in zip((8, 16, 32), secs)}}

    # one stream per solve: the two independent solves of a step run
    # concurrently (the GPU is mostly idle during one solve's one-CTA
    # Rayleigh-Ritz eigenproblems), as the serving loop runs its requests
    streams = {m: torch.cuda.Stream() for m in METHODS}

    def make(method, precision, st=None):
        p = kl.params(geometry=args["geometry"], degree=args["p"], elems=args["elems"], kernel=args["kernel"],
                      sigma=args["sigma"], L=args["L"], geo=geo, method=method, precision=precision, block_k=ks[method],
                      seed=2101 + 7919 * rank)
        return kl.kl_create(p, st if st is not None else stream)

    handles = {m: make(m, a.precision, streams[m]) for m in METHODS}
    # in the concurrent step each solve's pairwise product leaves SHARED_SMS
    # SMs to the other stream, whose short kernels would otherwise wait for
    # the end of every product (a persistent grid over all SMs holds them all)
    for m in METHODS:
        kl.kl_set_shared_sms(handles[m], SHARED_SMS)
    N = kl.kl_dims(handles["galerkin"])[0]
    lam = {m: np.zeros(M) for m in METHODS}
    res = {m: np.zeros(M) for m in METHODS}
    Vd = {m: torch.empty((M, N), dtype=torch.float64, device="cuda") for m in METHODS}
    infos = {m: kl.kl_solve_info() for m in METHODS}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    def solve(method):
        rc = kl.kl_eigs(handles[method], M, 0.0, lam[method], Vd[method], N, 1, res[method], infos[method])
        if rc != 0:
            raise RuntimeError(f"{method} solve returned status {rc}")

    def step_concurrent():
        """Both solves on their own streams from two host threads (ctypes
        releases the GIL), timed on the device: a start event both streams
        wait on, an end event after both."""
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        es = {m: torch.cuda.Event(enable_timing=True) for m in METHODS}
        ee = {m: torch.cuda.Event(enable_timing=True) for m in METHODS}
        e0.record(stream)
        for m in METHODS:
            streams[m].wait_event(e0)
            es[m].record(streams[m])
        errors = []

        def run(m):
            try:
                solve(m)
            except Exception as exc:  # re-raised on the main thread
                errors.append(exc)

        threads = [threading.Thread(target=run, args=(m,)) for m in METHODS]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
        for m in METHODS:
            ee[m].record(streams[m])
            stream.wait_event(ee[m])
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), {m: es[m].elapsed_time(ee[m]) for m in METHODS}

    def step_sequential():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        es = {m: torch.cuda.Event(enable_timing=True) for m in METHODS}
        ee = {m: torch.cuda.Event(enable_timing=True) for m in METHODS}
        e0.record(stream)
        for m in METHODS:
            streams[m].wait_event(e0)
            es[m].record(streams[m])
            solve(m)
            ee[m].record(streams[m])
        for m in METHODS:
            stream.wait_event(ee[m])
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), {m: es[m].elapsed_time(ee[m]) for m in METHODS}

    if a.profile_step:
        for m in METHODS:
            solve(m)
        torch.cuda.synchronize()
        for m in METHODS:
            kl.kl_destroy(handles[m])
        return

    for _ in range(max(3, a.warmup)):
        step_concurrent()
    torch.cuda.synchronize()

    launches0 = sum(kl.kl_launch_count(handles[m]) for m in METHODS)
    step_ms, solve_ms, seq_ms, alone_ms = [], {m: [] for m in METHODS}, [], {m: [] for m in METHODS}
    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_region = time.perf_counter()
    for _ in range(a.steps):
        flush.zero_()  # L2 flush between timed steps (outside the step events)
        torch.cuda.synchronize()
        t, per = step_concurrent()
        step_ms.append(t)
        for m in METHODS:
            solve_ms[m].append(per[m])
    # the same steps with the solves one after the other; the pairwise
    # kernel's per-launch durations for the roofline are taken here (no
    # other stream shares the GPU)
    # alone, a solve's pairwise product takes every SM (one untimed step
    # captures the graphs of that grid)
    for m in METHODS:
        kl.kl_set_shared_sms(handles[m], 0)
    step_sequential()
    for m in METHODS:
        kl.kl_profile_enable(handles[m], True)
    for _ in range(a.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t, per = step_sequential()
        seq_ms.append(t)
        for m in METHODS:
            alone_ms[m].append(per[m])
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    region_s = time.perf_counter() - t_region
    clk = clocks.stop()
    launches = sum(kl.kl_launch_count(handles[m]) for m in METHODS) - launches0
    prof = {}
    method_units = {}  # kernel evaluations counted as the method defines its work
    for m in METHODS:
        _, S_m, T_m = kl.kl_dims(handles[m])
        for name, st in kl.kl_profile_read(handles[m]).items():
            acc = prof.setdefault(name, dict(launches=0, ms=0.0, units=0.0))
            for key in acc:
                acc[key] += st[key]
            # Galerkin: Gamma over one point set is symmetric, N~(N~+1)/2
            # distinct pairs per vector block (what the symmetric class
            # counts already); collocation: every pair
            sym = (S_m + 1) / (2.0 * S_m) if (m == "galerkin" and S_m == T_m and not name.endswith("_sym")) else 1.0
            method_units[name] = method_units.get(name, 0.0) + st["units"] * sym
        kl.kl_profile_enable(handles[m], False)
    ms_step = float(np.mean(step_ms))
    if dist is not None:
        ms_step = max_over_ranks(ms_step, dist, "cuda")

    # ---- FP64 GPU solves of the same step (the reference precision) ----
    fp64 = {}
    if not a.no_fp64:
        for m in METHODS:
            h64 = make(m, "fp64")
            lam64 = np.zeros(M)
            info64 = kl.kl_solve_info()
            kl.kl_eigs(h64, M, 0.0, lam64, None, N, 0, None, info64)  # warm-up
            t64, _ = _timed_solve(kl, torch, stream, h64, M, 0.0, lam64, info64)
            err = _lam_err(lam[m], lam64)
            # the same FP64 solve stopped at the mixed solve's residual
            # tolerance (1e-6): the time an FP64 solve needs for the accuracy
            # the metric asks for (lambda error <= 1e-5)
            lam64m = np.zeros(M)
            info64m = kl.kl_solve_info()
            t64m, _ = _timed_solve(kl, torch, stream, h64, M, 1e-6, lam64m, info64m)
            fp64[m] = dict(s=t64, applies=info64.applies, lam=lam64.tolist(),
                           lam_rel_err=err.tolist(), max_lam_rel_err=float(err.max()),
                           matched_tol=dict(tol=1e-6, s=t64m, applies=info64m.applies,
                                            max_lam_rel_err=float(_lam_err(lam64m, lam64).max())))
            kl.kl_destroy(h64)

    # ---- serving: continuous batching of a seeded request stream ----
    serving = None
    if not a.no_serve and rank == 0 and world == 1:
        serving = _serve_leg(a, kl, stream)

    # ---- end to end through the C ABI with host buffers ----
    e2e_ms = []
    lam_h = np.zeros(M)
    V_h = np.zeros((M, N))
    h2d = 0
    for _ in range(2):
        t0 = time.perf_counter()
        for m in METHODS:
            p = kl.params(geometry=args["geometry"], degree=args["p"], elems=args["elems"], kernel=args["kernel"],
                          sigma=args["sigma"], L=args["L"], geo=geo, method=m, precision=a.precision, block_k=ks[m])
            h = kl.kl_create(p, stream)
            h2d_m, _ = kl.kl_memory(h)
            kl.kl_eigs(h, M, 0.0, lam_h, V_h, N, 0)
            kl.kl_destroy(h)
            h2d += h2d_m
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    h2d //= 2
    d2h = len(METHODS) * (M * N * 8 + M * 8)

    # ---- roofline of the dominant kernel ----
    fp32_fma, ex2, fp64_fma = kl.kl_measure_peaks()
    pair_name = max(prof, key=lambda n: prof[n]["ms"]) if prof else None
    roof = None
    if pair_name:
        st = prof[pair_name]
        achieved = st["units"] / (st["ms"] * 1e-3) / 1e9  # Gpair/s
        # ALU roof of one kernel evaluation: special-function ops (ex2, and
        # sqrt for the Euclidean kernels) on the MUFU pipe and the FP32 ops
        # the formula needs on the FP32 pipe (coordinate differences, the
        # argument, the Matern polynomial); the split and the products are
        # this design's own work and are not counted
        mufu_per_pair, fp32_per_pair = ALU_OPS_PER_PAIR[args["kernel"]]
        peak_mufu = ex2 / mufu_per_pair / 1e9
        peak_fp32 = fp32_fma / fp32_per_pair / 1e9
        peak = min(peak_mufu, peak_fp32)
        achieved_m = method_units[pair_name] / (st["ms"] * 1e-3) / 1e9
        roof = {"bound": "alu", "kernel": pair_name, "achieved": achieved, "peak": peak, "unit": "Gpair/s",
                "frac": achieved / peak, "traffic": _recorded_traffic(pair_name),
                "achieved_method_count": achieved_m, "frac_method_count": achieved_m / peak,
                "method_count": "Galerkin pairs counted once per symmetric pair, N~(N~+1)/2 (the symmetric class "
                                "pair_tc_bf16_sym evaluates each once: its achieved is that count; the dense classes "
                                "evaluate all N~^2); collocation N N_eN_q",
                "peak_basis": f"min(measured MUFU ex2 {ex2 / 1e12:.2f} T/s / {mufu_per_pair} per pair, measured FP32 "
                              f"{fp32_fma / 1e12:.1f} T op/s / {fp32_per_pair} per pair); FP64 FMA "
                              f"{fp64_fma / 1e12:.2f} T/s",
                "launches": st["launches"], "ms": st["ms"], "pairs": st["units"]}
    # ---- the annulus workloads (solve times, FP64 comparison, pairwise roofline) ----
    configs = None
    if not a.no_configs and rank == 0 and a.workload == WORKLOAD:
        configs = _configs_leg(a, kl, stream, (fp32_fma, ex2, fp64_fma))

    # ---- K-L field sampling with the computed eigenpairs (not in the step) ----
    sampling = _sampling_leg(kl, handles, streams, lam, Vd, N, M, args, fp64_fma) if rank == 0 else None

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu and a.workload == WORKLOAD:
        # the GPU on the same sample problem (same precision and block size as
        # the step), second solve of each handle, CUDA events; before the
        # oracle, whose BLAS threads would compete with the solver's host thread
        gpu_sample = {}
        for m in METHODS:
            ps = kl.params(geometry=args["geometry"], degree=args["p"], elems=(CPU_SAMPLE_ELEMS,) * 3,
                           kernel=args["kernel"], sigma=args["sigma"], L=args["L"], geo=geo, method=m,
                           precision=a.precision, block_k=k, seed=2101)
            hs = kl.kl_create(ps, stream)
            lam_s = np.zeros(M)
            for _ in range(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                kl.kl_eigs(hs, M, 0.0, lam_s, None, 0, 0)
                e1.record(stream)
                e1.synchronize()
            gpu_sample[m] = e0.elapsed_time(e1) / 1e3
            kl.kl_destroy(hs)
        v, per, cores = _oracle_sample(CPU_SAMPLE_ELEMS)
        cpu = {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
               "sample": _sample_text(CPU_SAMPLE_ELEMS, per),
               "gpu_same_sample_s": sum(gpu_sample.values()), "gpu_same_sample_per_method_s": gpu_sample,
               "oracle_over_gpu_same_sample": v / sum(gpu_sample.values())}

    p50 = {m: float(np.percentile(solve_ms[m], 50)) for m in METHODS}
    p99 = {m: float(np.percentile(solve_ms[m], 99)) for m in METHODS}
    p50a = {m: float(np.percentile(alone_ms[m], 50)) for m in METHODS}
    p99a = {m: float(np.percentile(alone_ms[m], 99)) for m in METHODS}
    line = {
        "metric": METRIC,
        "value": ms_step / 1e3 if world == 1 else ms_step / 1e3,
        "unit": "s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": max(3, a.warmup),
        "ms_per_step": ms_step,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 kernel tiles, split-bf16 tcgen05 products, f64 solver" if a.precision == "bf16" else a.precision,
        "data": "synthetic",
        "config": {"workload": a.workload, "N": N, "M": M, "k": (dict(ks) if a.autotune else k), "methods": list(METHODS),
                   **({"autotune": tuned} if a.autotune else {}),
                   "precision": a.precision, "l2": "flushed between steps (256 MB write)",
                   "step": "the Galerkin and the collocation solve run concurrently on two streams",
                   "shared_sms": SHARED_SMS,
                   "parallelism": "replicas" if world > 1 else "single"},
        "ms_per_step_sequential": float(np.mean(seq_ms)),
        "solve_ms_p50": p50, "solve_ms_p99": p99,
        "solve_ms_p50_alone": p50a, "solve_ms_p99_alone": p99a,
        "fp64_gpu": {m: {kk: v for kk, v in fp64[m].items() if kk != "lam"} for m in fp64},
        "speedup_vs_fp64": ({m: fp64[m]["s"] * 1e3 / p50a[m] for m in fp64} if fp64 else None),
        "speedup_vs_fp64_matched_tol": ({m: fp64[m]["matched_tol"]["s"] * 1e3 / p50a[m] for m in fp64}
                                        if fp64 else None),
        "configs": configs,
        "lam": {m: lam[m].tolist() for m in METHODS},
        "applies": {m: infos[m].applies for m in METHODS},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": float(np.median(e2e_ms)) / 1e3, "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "serving": serving,
        "sampling": sampling,
        "gpu_launches": int(launches),
        "clocks": clk,
        "region_s": region_s,
    }
    for m in METHODS:
        kl.kl_destroy(handles[m])
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def run_accuracy(a):
    """Accuracy versus time in the manner of Sec. 4 (Figs. 4-6): the mixed
    precision solves of every method on h-refined unit-cube meshes (p = 2),
    their eigensolver time, and the mean / largest relative error of their
    first M eigenvalues against the reference, the standard Gauss-Legendre
    Galerkin solution in FP64 on the finest mesh (as the paper's reference is
    the standard Galerkin solution on its finest mesh)."""
    import numpy as np
    import torch
    import paper_2101_00629_gb300 as kl

    M, k = 20, 8
    L = {"gauss": 0.5}.get(a.accuracy_kernel, 1.0)
    elems = [int(x) for x in a.accuracy_elems.split(",")]
    stream = torch.cuda.current_stream()

    def solve(method, e, precision, reps=2):
        p = kl.params(geometry="cube", degree=2, elems=(e, e, e), kernel=a.accuracy_kernel, sigma=1.0, L=L,
                      method=method, precision=precision, block_k=k, seed=2101)
        h = kl.kl_create(p, stream)
        N = kl.kl_dims(h)[0]
        lam = np.zeros(M)
        ms = None
        for _ in range(reps):  # the first solve captures the graphs
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = kl.kl_eigs(h, M, 0.0, lam, None, 0, 0)
            e1.record(stream)
            e1.synchronize()
            if rc not in (0, 1):
                raise RuntimeError(f"{method} {e}^3 {precision}: status {rc}")
            ms = e0.elapsed_time(e1)
        kl.kl_destroy(h)
        return N, ms, lam.copy()

    N_ref, ref_ms, ref = solve("galerkin_std", max(elems), "fp64", reps=1)
    points = []
    for method in ("galerkin", "collocation", "galerkin_std"):
        for e in elems:
            N, ms, lam = solve(method, e, a.precision)
            err = np.abs(lam - ref) / np.abs(ref)
            points.append({"method": method, "elems": e, "N": N, "solve_ms": round(ms, 3),
                           "mean_rel_err": float(err.mean()), "max_rel_err": float(err.max())})
    print(json.dumps({
        "mode": "accuracy", "kernel": a.accuracy_kernel, "L": L, "sigma": 1.0, "p": 2, "M": M, "k": k,
        "precision": a.precision,
        "reference": {"method": "galerkin_std", "precision": "fp64", "elems": max(elems), "N": N_ref,
                      "solve_ms": round(ref_ms, 3)},
        "points": points,
    }))


# Sec. 4 benchmark cases on the half annular cylinder: the meshes reproduce the
# dof counts of Tables 1-2 (tests/golden/half_cylinder_dofs.txt); the
# dimensions are not printed, these give elements of about the printed mesh
# size h; correlation length 5 (Fig. 1 caption).
PAPER_GEO = (27.5, 30.5, 23.0)
PAPER_L = 5.0
PAPER_EX1 = [(1, (32, 1, 8)), (2, (28, 2, 15)), (3, (32, 2, 18)), (4, (38, 2, 21)), (5, (42, 3, 23))]
PAPER_EX2 = [(1, 2), (2, 3), (3, 4), (4, 5), (5, 6)]


def run_accuracy_paper(a):
    """Example 1 (exponential kernel, h-refinement, p = 2, split-BF16 solves)
    and Example 2 (Gaussian kernel, k-refinement on the Case 1 mesh,
    p = 2..6, FP64 solves): eigensolver time and error of the first 20
    eigenvalues of both methods against a standard Gauss-Legendre Galerkin
    reference (Example 1: twice as fine as Case 5; Example 2: p = 6)."""
    import numpy as np
    import torch
    import paper_2101_00629_gb300 as kl

    M, k = 20, 8
    stream = torch.cuda.current_stream()

    def solve(method, p, elems, kernel, precision, reps=2):
        prm = kl.params(geometry="half_annulus", degree=p, elems=elems, kernel=kernel, sigma=1.0, L=PAPER_L,
                        method=method, precision=precision, block_k=k, seed=2101)
        prm.geo[0], prm.geo[1], prm.geo[2] = PAPER_GEO
        h = kl.kl_create(prm, stream)
        dims = kl.kl_dims(h)
        lam = np.zeros(M)
        ms = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = kl.kl_eigs(h, M, 0.0, lam, None, 0, 0)
            e1.record(stream)
            e1.synchronize()
            if rc not in (0, 1):
                raise RuntimeError(f"{method} p={p} {elems} {precision}: status {rc}")
            ms = e0.elapsed_time(e1)
        kl.kl_destroy(h)
        return dims, ms, lam.copy()

    out = {"mode": "accuracy", "study": "paper", "geometry": "half_annulus", "geo": PAPER_GEO, "L": PAPER_L,
           "sigma": 1.0, "M": M, "k": k, "examples": {}}
    fine = tuple(2 * n for n in PAPER_EX1[-1][1])
    rdims, rms, ref1 = solve("galerkin_std", 2, fine, "exp", a.precision, reps=1)
    pts = []
    for case, elems in PAPER_EX1:
        for method in ("galerkin", "collocation"):
            dims, ms, lam = solve(method, 2, elems, "exp", a.precision)
            err = np.abs(lam - ref1) / np.abs(ref1)
            pts.append({"case": case, "method": method, "elems": elems, "N": dims[0], "points": dims[1],
                        "solve_ms": round(ms, 3), "mean_rel_err": float(err.mean()), "max_rel_err": float(err.max())})
    out["examples"]["1"] = {"kernel": "exp", "p": 2, "precision": a.precision, "points": pts,
                            "reference": {"method": "galerkin_std", "precision": a.precision, "elems": fine,
                                          "N": rdims[0], "solve_ms": round(rms, 3)}}
    mesh2 = PAPER_EX1[0][1]
    rdims, rms, ref2 = solve("galerkin_std", 6, mesh2, "gauss", "fp64", reps=1)
    pts = []
    for case, p in PAPER_EX2:
        for method in ("galerkin", "collocation"):
            dims, ms, lam = solve(method, p, mesh2, "gauss", "fp64")
            err = np.abs(lam - ref2) / np.abs(ref2)
            pts.append({"case": case, "method": method, "p": p, "N": dims[0], "points": dims[1],
                        "solve_ms": round(ms, 3), "mean_rel_err": float(err.mean()), "max_rel_err": float(err.max())})
    out["examples"]["2"] = {"kernel": "gauss", "elems": mesh2, "precision": "fp64", "points": pts,
                            "reference": {"method": "galerkin_std", "precision": "fp64", "p": 6, "N": rdims[0],
                                          "solve_ms": round(rms, 3)}}
    print(json.dumps(out))


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
        return
    if a.accuracy:
        if a.accuracy_study == "paper":
            run_accuracy_paper(a)
        else:
            run_accuracy(a)
        return
    run_gpu(a)


if __name__ == "__main__":
    main()
