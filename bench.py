"""Benchmark of the BLDTT compute phase on GB300.

Workload: 1E6 particles uniform in [-1,1]^3 (targets = sources), charges
uniform in [-1,1], Coulomb kernel, n=8, theta=0.7, leaves of 2000, FP32-bulk
kernel evaluations (FP64 accumulation).  One step is the whole hot path:
bldtt_setup (both trees, traversal, work lists) and bldtt_compute (upward
pass, PP/PC/CP/CC interactions, downward pass, potentials in input order) on
inputs already resident in device memory.  The plain FP64 BLDTT is run on the
same inputs to check the rel-l2 error (<= 1e-6) and timed as the FP64
comparator.

Multi-GPU: one process per GPU (torchrun).  Every rank sets up the same plan
and computes one shard of the target leaves (bldtt_compute_shard); the shards'
potentials are summed over ranks (NCCL all-reduce of zero-filled buffers), so
the job solves the one problem of the workload and `value` is its targets per
second (strong scaling).  The batched and 1E8 workloads run one replica per
rank (weak scaling).

`--impl reference` times the CPU oracle (FP64, numpy) instead, on a bounded
sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "targets/sec at rel. L2 error ≤1e-6 vs plain FP64 BLDTT, 1 GB300; % FP32 peak"
UNIT = "targets/s"
WORKLOAD = "uniform_n1e6"
FLOPS_PER_EVAL = {0: 20.0, 1: 28.0}   # Coulomb, Yukawa (stated flop counts)


def max_over_ranks(ms: float, dist=None) -> float:
    """The slowest rank's time (all ranks get it); ms itself for one process.
    NCCL groups reduce on the GPU, gloo groups on the CPU."""
    if dist is None:
        return ms
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(targets_per_rank: int, steps: int, world: int, total_ms: float) -> float:
    """Whole-job targets/s: every rank solves its own replica (weak scaling),
    timed by the slowest rank."""
    return targets_per_rank * steps * world / (total_ms / 1000.0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["uniform_n1e6", "unequal_yukawa", "plain_fp64_n2e4", "uniform_n1e8",
                             "batched_512"],
                    help="workload to time (default: the 1E6 uniform Coulomb workload)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparator timing")
    ap.add_argument("--pass-engine", default="default", choices=["default", "simt", "tensor"],
                    help="engine of the FP32 leaf contractions (default: the library's per-pass "
                         "choice, SIMT upward and tensor cores downward)")
    return ap.parse_args()


def workload(name=WORKLOAD):
    from paper_2012_06925_gb300 import workloads as W
    cfg = dict(W.CONFIGS[name])
    cfg["name"] = name
    tgt, src, q = W.make_problem(cfg["kind"], cfg["M"], cfg["N"], seed=cfg["seed"],
                                 sources_kind=cfg.get("sources_kind"))
    kw = dict(kernel=cfg["kernel"], kappa=cfg["kappa"], n=cfg["n"], theta=cfg["theta"],
              N0=cfg["N0"], M0=cfg["M0"])
    return cfg, tgt, src, q, kw


def config_dict(cfg):
    kern = "Coulomb" if cfg["kernel"] == 0 else f"Yukawa kappa={cfg['kappa']}"
    if cfg["N"] is None:
        sets = f"M=N={cfg['M']:.0e} {cfg['kind']} in [-1,1]^3, targets=sources"
    else:
        sets = (f"M={cfg['M']:.0e} {cfg['kind']} targets, N={cfg['N']:.0e} "
                f"{cfg.get('sources_kind') or cfg['kind']} sources")
    return {"workload": f"{cfg['name']}: {sets}, charges U[-1,1], {kern}, n={cfg['n']}, "
                        f"theta={cfg['theta']}, N0=M0={cfg['N0']}, FP32-bulk evaluation with FP64 "
                        f"accumulation",
            "M": cfg["M"], "N": cfg["N"] or cfg["M"], "n": cfg["n"], "theta": cfg["theta"],
            "leaf": cfg["N0"], "kernel": "coulomb" if cfg["kernel"] == 0 else "yukawa",
            "l2": "flushed between timed steps (256 MiB write)"}


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, multiprocessing, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
import oracle as O
from paper_2012_06925_gb300 import workloads as W
cfg = W.CONFIGS[%(wl)r]
tgt, _, q = W.make_problem(cfg["kind"], cfg["M"], seed=cfg["seed"])
kw = dict(kernel=cfg["kernel"], kappa=cfg["kappa"], n=cfg["n"], theta=cfg["theta"],
          N0=cfg["N0"], M0=cfg["M0"])
t0 = time.perf_counter()
samp = O.SampledBLDTT(tgt, tgt, q, **kw)
setup_s = time.perf_counter() - t0
leaves = samp.tt.leaves()


def one(k):
    leaf = leaves[k %% len(leaves)]
    idx = samp.tt.perm[np.arange(samp.tt.begin[leaf], samp.tt.end[leaf])]
    t1 = time.perf_counter()
    samp.potentials(idx)
    return int(idx.size), time.perf_counter() - t1


# Workers are forked from this process, which never touches a GPU; each is
# one single-threaded oracle on one host core.
with multiprocessing.get_context("fork").Pool(%(cores)d) as pool:
    for group in %(groups)r:
        t1 = time.perf_counter()
        res = pool.map(one, group, chunksize=1)
        print(json.dumps(dict(setup_s=setup_s, wall_s=time.perf_counter() - t1,
                              sample=sum(r[0] for r in res), leaves=len(res),
                              M=int(cfg["M"]))), flush=True)
"""


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rates(groups, cores=None):
    """Time the oracle on whole target leaves, one group of leaves at a time
    (leaf indices in tree order), the leaves of a group in parallel, one
    single-threaded oracle process per host core.  The trees, the traversal
    and the upward pass are built once, for all M particles, and charged to
    each group pro rata (its targets / M): per target the oracle then sums the
    PP/PC entries of the target's cluster chain and interpolates the chain's
    CP/CC proxy potentials, which a whole leaf shares."""
    cores = cores or host_cores()
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET % dict(root=ROOT, wl=WORKLOAD, groups=[list(g) for g in groups],
                                 cores=cores)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed:\n" + r.stderr[-2000:])
    out = []
    for ln in r.stdout.strip().splitlines():
        d = json.loads(ln)
        t = d["wall_s"] + d["setup_s"] * d["sample"] / d["M"]
        out.append(dict(value=d["sample"] / t, unit=UNIT, cores=cores, kind="oracle",
                        sample=(f"{d['leaves']} whole target leaves ({d['sample']} targets) of the "
                                f"{WORKLOAD} workload, one per host core, in parallel (FP64 numpy "
                                f"oracle, one thread per process): per-target PP/PC along the "
                                f"cluster chain plus the chain's CP/CC proxy potentials "
                                f"({d['wall_s']:.2f} s); trees, traversal and upward pass for all "
                                f"{d['M']:.0e} particles ({d['setup_s']:.1f} s, once) charged pro "
                                f"rata"),
                        seconds=t))
    if len(out) != len(groups):
        raise RuntimeError("oracle timing printed %d of %d groups" % (len(out), len(groups)))
    return out


def leaf_groups(count, cores):
    """count groups of `cores` distinct leaf indices each."""
    return [list(range(k * cores, (k + 1) * cores)) for k in range(count)]


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2012_06925_gb300 import workloads as W
    cfg = dict(W.CONFIGS[WORKLOAD])
    cfg["name"] = WORKLOAD
    # one leaf per host core per step (different leaves each step), the
    # oracle's set-up once
    cores = host_cores()
    rates = oracle_rates(leaf_groups(args.warmup + args.steps, cores), cores)[args.warmup:]
    value = statistics.median([r["value"] for r in rates])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.median([r["seconds"] for r in rates]),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(cfg),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": rates[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = [r for r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [nm for k, nm in enumerate(names) if any(r[5 + k] == "Active" for r in rows)]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def code_hash(*paths):
    """sha256 of source files' code: // comments, blank lines and indentation
    removed, so that editing a comment does not change it."""
    import hashlib
    lines = []
    for path in paths:
        with open(path) as f:
            for line in f:
                code = line.split("//", 1)[0].strip()
                if code:
                    lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def _kernel_header_code(path):
    """The parts of the shared header that the interaction kernel compiles
    with: its constants and its device helper functions."""
    keep, in_fn = [], False
    with open(path) as f:
        for line in f:
            code = line.split("//", 1)[0].rstrip()
            if code.lstrip().startswith("constexpr"):
                keep.append(code.strip())
            if "__device__" in code:
                in_fn = True
            if in_fn:
                if code.strip():
                    keep.append(code.strip())
                if code == "}":
                    in_fn = False
    return "\n".join(keep)


def interact_code_hash():
    """sha256 of the interaction kernel's code: interact.cu (code lines) and
    the constants and device helpers of internal.cuh."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2012_06925_gb300", "csrc")
    h = hashlib.sha256(code_hash(os.path.join(csrc, "interact.cu")).encode())
    h.update(_kernel_header_code(os.path.join(csrc, "internal.cuh")).encode())
    return h.hexdigest()


def interact_traffic():
    """DRAM bytes per launch of the interaction kernel from the committed ncu
    summary, if it was taken on the current kernel code."""
    path = os.path.join(ROOT, "profiles", "interact_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("interact_code_sha256") == interact_code_hash():
            return d.get("dram_bytes_per_launch_full_size")
    except (OSError, ValueError):
        pass
    return None


def pipe_rates(stream) -> dict:
    """Measured lanes per clock per SM of the FP32 FMA pipe (scalar and packed),
    MUFU rsqrt and exp2 and FP64 FMA, from the benchmark's own probe library
    (libbldtt_pipes.so, not part of libbldtt.so)."""
    import ctypes

    import numpy as np

    from paper_2012_06925_gb300 import build as builder
    lib = ctypes.CDLL(builder.build_pipes())
    lib.pipes_rates.restype = ctypes.c_int
    lib.pipes_rates.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    lib.pipes_last_error.restype = ctypes.c_char_p
    out = np.zeros(5, dtype=np.float64)
    rc = lib.pipes_rates(out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         ctypes.c_void_p(stream.cuda_stream if stream is not None else 0))
    if rc != 0:
        raise RuntimeError("pipe probe failed: " + lib.pipes_last_error().decode())
    return dict(ffma=out[0], ffma2_lanes=out[1], mufu_rsqrt=out[2], mufu_ex2=out[3], dfma=out[4])


def relative_errors(reference, approx):
    """(rel-l2, max-norm) of approx against reference: ||d||_2/||ref||_2 and
    ||d||_inf/||ref||_inf."""
    import numpy as np
    d = np.asarray(approx, dtype=np.float64) - np.asarray(reference, dtype=np.float64)
    ref = np.asarray(reference, dtype=np.float64)
    return (float(np.sqrt(np.sum(d * d) / np.sum(ref * ref))),
            float(np.max(np.abs(d)) / np.max(np.abs(ref))))


def gather_potentials(phi, dist):
    """Every rank's potentials into every rank's phi: each rank computed its
    own shard of the target leaves into a zero-filled phi, so the sum over
    ranks is exact (x + 0 = x) and equals the one-GPU result."""
    if dist is not None:
        dist.all_reduce(phi, op=dist.ReduceOp.SUM)
    return phi


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2012_06925_gb300 import binding as B
    from paper_2012_06925_gb300 import build as builder

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    builder.build()
    B.load_library()

    cfg, tgt, src, q, kw = workload(args.workload)
    M = tgt.shape[1]
    N = src.shape[1]
    same = src is tgt
    dt = torch.from_numpy(tgt).cuda()
    ds = dt if same else torch.from_numpy(src).cuda()
    dq = torch.from_numpy(q).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    st_engines = [None, None]

    def step(precision, phi):
        """Set-up and compute of the whole problem: one GPU computes it all;
        with N ranks each computes its shard of the target leaves and the
        shards' potentials are gathered (the job's one exchange)."""
        plan = B.Plan(dt, ds, dq, precision=precision, stream=stream, **kw)
        if precision == B.FP32_BULK:
            if args.pass_engine != "default":
                e = B.PASS_TENSOR if args.pass_engine == "tensor" else B.PASS_SIMT
                plan.set_pass_engine(e, e)
            st_engines[:] = [plan.pass_engine_used(0), plan.pass_engine_used(1)]
        if dist is None:
            plan.compute(phi, stream=stream)
        else:
            phi.zero_()
            plan.compute_shard(rank, world, phi, stream=stream)
            gather_potentials(phi, dist)
        return plan

    # Accuracy gate: FP32-bulk against the plain FP64 BLDTT on the same inputs.
    phi64 = torch.empty(M, dtype=torch.float64, device="cuda")
    phi32 = torch.empty(M, dtype=torch.float64, device="cuda")
    p64 = step(B.FP64, phi64)
    p64.check_error()
    st64 = p64.stats()
    p64.close()
    p32 = step(B.FP32_BULK, phi32)
    p32.check_error()
    p32.close()
    a64, a32 = phi64.cpu().numpy(), phi32.cpu().numpy()
    rel_l2, max_norm = relative_errors(a64, a32)
    # The workload's own error measure: both precisions against the FP64
    # direct sum (Eq. (1), on the device) at 2000 seeded sampled targets.
    samp = np.sort(np.random.default_rng(7).choice(M, size=min(M, 2000), replace=False))
    direct = B.direct_sum(torch.from_numpy(np.ascontiguousarray(tgt[:, samp])).cuda(), ds, dq,
                          kw["kernel"], kw["kappa"]).cpu().numpy()
    e64, m64 = relative_errors(direct, a64[samp])
    e32, m32 = relative_errors(direct, a32[samp])
    vs_direct = {"samples": int(samp.size), "seed": 7,
                 "fp32_bulk": {"rel_l2": e32, "max_norm": m32},
                 "fp64": {"rel_l2": e64, "max_norm": m64}}

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step(B.FP32_BULK, phi32).close()

    barrier()
    times, st_list = [], []
    with ClockSampler(local) as clocks:
        for _ in range(args.steps):
            flush.fill_(float(len(times)))                   # evict L2 between steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan = step(B.FP32_BULK, phi32)
            e1.record(stream)
            st_list.append(plan.stats())                     # synchronises
            plan.close()
            times.append(e0.elapsed_time(e1))
    barrier()
    total_ms = sum(times)
    total_ms = max_over_ranks(total_ms, dist)
    # End to end through the public API from pinned host buffers: one GPU
    # calls bldtt_solve_host (copies in, set-up, compute, potentials out); N
    # ranks copy the inputs in, set up, compute their shards, gather the
    # potentials and copy them out.
    ht = torch.from_numpy(tgt).pin_memory()
    hs = ht if same else torch.from_numpy(src).pin_memory()
    hq = torch.from_numpy(q).pin_memory()
    host_phi = torch.empty(M, dtype=torch.float64).pin_memory()
    e2e_times = []
    import ctypes
    lib = B.load_library()
    st_buf = B.Stats()
    for i in range(1 + max(1, min(3, args.steps))):
        flush.fill_(float(i))
        barrier()
        t0 = time.perf_counter()
        if dist is None:
            rc = lib.bldtt_solve_host(ctypes.cast(ht.data_ptr(), ctypes.POINTER(ctypes.c_double)), M,
                                      ctypes.cast(hs.data_ptr(), ctypes.POINTER(ctypes.c_double)), N,
                                      ctypes.cast(hq.data_ptr(), ctypes.POINTER(ctypes.c_double)),
                                      kw["kernel"], kw["kappa"], kw["n"], kw["theta"], kw["N0"],
                                      kw["M0"], B.FP32_BULK,
                                      ctypes.cast(host_phi.data_ptr(), ctypes.POINTER(ctypes.c_double)),
                                      ctypes.byref(st_buf))
            B._check(rc)
        else:
            dt2 = ht.cuda(non_blocking=True)
            ds2 = dt2 if same else hs.cuda(non_blocking=True)
            dq2 = hq.cuda(non_blocking=True)
            plan = B.Plan(dt2, ds2, dq2, precision=B.FP32_BULK, stream=stream, **kw)
            phi32.zero_()
            plan.compute_shard(rank, world, phi32, stream=stream)
            gather_potentials(phi32, dist)
            host_phi.copy_(phi32, non_blocking=True)
            torch.cuda.synchronize()
            plan.close()
        t1 = time.perf_counter()
        if i > 0:
            e2e_times.append(t1 - t0)
    e2e_s = max_over_ranks(statistics.median(e2e_times) * 1000.0, dist) / 1000.0
    e2e = {"value": M / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(ht.numel() * 8 + (0 if same else hs.numel() * 8) + hq.numel() * 8),
           "d2h_bytes_per_step": int(M * 8), "seconds": e2e_s}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    st = st_list[-1]
    value = job_rate(M, args.steps, 1, total_ms)      # one problem, shared by all ranks
    ms_interact = statistics.mean(s["ms_interact"] for s in st_list)
    evals = st["computed_evaluations"]                 # this rank's work items
    flops = FLOPS_PER_EVAL.get(kw["kernel"], 20.0) * evals
    achieved = flops / (ms_interact / 1000.0) / 1e12
    props = torch.cuda.get_device_properties(local)
    sm_max = measured_peaks().get("sm_max_mhz", 2070.0)
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    csum = clocks.summary()
    launches = sum(s["launches_setup"] + s["launches_compute"] for s in st_list)
    peaks = measured_peaks()
    load_mhz = peaks.get("clocks_under_load", {}).get("sm_mhz_median")

    # Issue ceilings beside the peak, from the library's pipe microbenchmark
    # (operations per clock per SM).  Per Coulomb evaluation the packed path
    # issues 3.5 FP32x2 instructions (7 lanes) and one MUFU.RSQ; Yukawa adds
    # one MUFU.EX2 and two lanes.
    rates = pipe_rates(stream)
    sms = props.multi_processor_count
    clock = (csum.get("sm_mhz") or sm_max) * 1e6
    fma_lanes_per_eval = 7.0 if kw["kernel"] == 0 else 9.0
    mufu_clk_per_eval = 1.0 / rates["mufu_rsqrt"] + (0.0 if kw["kernel"] == 0 else 1.0 / rates["mufu_ex2"])
    ceilings = {
        "unit": "evaluations/clk/SM",
        "fp32_pipe": rates["ffma2_lanes"] / fma_lanes_per_eval,
        "mufu": 1.0 / mufu_clk_per_eval,
        "achieved": evals / (ms_interact / 1000.0) / clock / sms,
        "measured_ops_per_clk_sm": {k: round(v, 2) for k, v in rates.items()},
    }
    ceilings["mufu_frac"] = ceilings["achieved"] / ceilings["mufu"]

    # Leaf passes: algorithmic bytes (32 B per particle read, the proxy arrays
    # of every cluster twice) and flops (2 n_p per particle), per phase time.
    np_ = (kw["n"] + 1) ** 3
    hbm = peaks.get("hbm_gbs", 6800.0)
    passes = {}
    for name, count, clusters in (("upward", N, st["num_source_clusters"]),
                                  ("downward", M, st["num_target_clusters"])):
        ms = st["ms_" + name]
        byts = 32.0 * count + 2.0 * 8.0 * np_ * clusters
        pflops = 2.0 * np_ * count
        passes[name] = {"ms": ms, "bytes": byts, "gbs": byts / (ms / 1000.0) / 1e9,
                        "hbm_frac": byts / (ms / 1000.0) / 1e9 / hbm,
                        "tflops": pflops / (ms / 1000.0) / 1e12,
                        "fp32_frac": pflops / (ms / 1000.0) / 1e12 / peak}

    # FP64 comparator: the plain FP64 BLDTT step, timed like the FP32 steps
    # over three steps (the accuracy-gate run above was its warm-up).
    fp64 = None
    if not args.no_fp64:
        ms64, int64 = [], []
        for i in range(3):
            flush.fill_(3.0 + i)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan = step(B.FP64, phi64)
            e1.record(stream)
            s64 = plan.stats()
            plan.close()
            ms64.append(e0.elapsed_time(e1))
            int64.append(s64["ms_interact"])
        fp64 = {"value": M * len(ms64) / (sum(ms64) / 1000.0), "unit": UNIT, "steps": len(ms64),
                "ms_per_step": sum(ms64) / len(ms64), "ms_per_step_each": ms64,
                "ms_interact": sum(int64) / len(int64)}

    cpu = None
    if world == 1 and not args.no_cpu_baseline and args.workload == WORKLOAD:
        try:
            cores = host_cores()
            cb = oracle_rates(leaf_groups(1, cores), cores)[0]
            cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        except Exception as exc:   # reported, not fatal
            cpu = {"value": None, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                   "sample": f"failed: {exc}"[:300]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(config_dict(cfg), parallelism=(f"target-leaf shards x{world}" if world > 1
                                                      else "one GPU")),
        "rel_l2_vs_fp64": rel_l2, "max_norm_vs_fp64": max_norm, "accuracy_ok": rel_l2 <= 1e-6,
        "rel_l2_vs_direct": vs_direct,
        "phases_ms": {"tree": st["ms_tree"], "lists": st["ms_lists"], "upward": st["ms_upward"],
                      "interact": st["ms_interact"], "downward": st["ms_downward"],
                      "compute": st["ms_compute"]},
        "interactions": {"PP": st["interactions"][0], "PC": st["interactions"][1],
                         "CP": st["interactions"][2], "CC": st["interactions"][3],
                         "executed_with_padding": st["executed_evaluations"]},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": interact_traffic(),
                     "kernel": f"k_interact<FP32,{'Coulomb' if kw['kernel'] == 0 else 'Yukawa'}>",
                     "flops_per_launch": flops, "ms_per_launch": ms_interact,
                     "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x "
                                   f"{sm_max:.0f} MHz",
                     "frac_at_sampled_clock": (achieved / peak * sm_max / csum["sm_mhz"])
                     if csum.get("sm_mhz") else None,
                     "frac_at_under_load_clock": (achieved / peak * sm_max / load_mhz)
                     if load_mhz else None,
                     "mufu_ceiling_frac": ceilings["mufu_frac"],
                     "ceilings": ceilings},
        "passes_roofline": passes,
        "pass_engines": {"upward": "tensor" if st_engines[0] == 1 else "simt",
                         "downward": "tensor" if st_engines[1] == 1 else "simt"},
        "fp64_plain": fp64,
        "speedup_vs_fp64": value / fp64["value"] if fp64 else None,
        "e2e": e2e, "gpu_launches": launches, "clocks": csum, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


BATCH = dict(count=512, seed=4, n=6, theta=0.7, N0=500, M0=500)


def run_gpu_batched(args):
    """512 independent problems (N log-uniform in [1E3, 1E5], half cube / half
    sphere surface, normal charges, Coulomb or Yukawa kappa ~ U[0.1, 2]) in one
    plan: a step is bldtt_setup_batch + bldtt_compute; the compute phase alone
    is also timed as replays of its captured CUDA graph after autotuning."""
    import numpy as np
    import torch

    from paper_2012_06925_gb300 import binding as B
    from paper_2012_06925_gb300 import build as builder
    from paper_2012_06925_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    builder.build()
    probs = W.batched_problems(count=BATCH["count"], seed=BATCH["seed"])
    pts = np.concatenate([p["points"] for p in probs], axis=1)
    q = np.concatenate([p["charges"] for p in probs])
    off = np.cumsum([0] + [p["points"].shape[1] for p in probs])
    kernels = [p["kernel"] for p in probs]
    kappas = [p["kappa"] for p in probs]
    M = pts.shape[1]
    dt = torch.from_numpy(pts).cuda()
    dq = torch.from_numpy(q).cuda()
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    kw = dict(n=BATCH["n"], theta=BATCH["theta"], N0=BATCH["N0"], M0=BATCH["M0"])

    def make(precision):
        return B.Plan.batch(dt, off, dt, off, dq, kernels, kappas, precision=precision,
                            stream=stream, **kw)

    with torch.cuda.stream(stream):
        phi64 = torch.empty(M, dtype=torch.float64, device="cuda")
        phi32 = torch.empty(M, dtype=torch.float64, device="cuda")
        p64 = make(B.FP64)
        p64.compute(phi64, stream=stream)
        p64.check_error()
        st64 = p64.stats()
        p64.close()
        p32 = make(B.FP32_BULK)
        layout = p32.autotune(phi32, stream=stream)
        p32.compute(phi32, stream=stream)
        p32.check_error()
        a64, a32 = phi64.cpu().numpy(), phi32.cpu().numpy()
        rel_l2 = float(np.sqrt(np.sum((a64 - a32) ** 2) / np.sum(a64 ** 2)))
        worst = max(float(np.sqrt(np.sum((a64[off[i]:off[i + 1]] - a32[off[i]:off[i + 1]]) ** 2)
                                  / np.sum(a64[off[i]:off[i + 1]] ** 2))) for i in range(len(probs)))
        # graph replays of the compute phase
        for _ in range(args.warmup):
            p32.compute_graph(phi32, stream)
        stream.synchronize()
        graph_ms = []
        for i in range(args.steps):
            flush.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p32.compute_graph(phi32, stream)
            e1.record(stream)
            e1.synchronize()
            graph_ms.append(e0.elapsed_time(e1))
        p32.close()
        # full steps: set-up + compute
        for _ in range(args.warmup):
            make(B.FP32_BULK).close()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        times, stats = [], []
        with ClockSampler(local) as clocks:
            for i in range(args.steps):
                flush.fill_(float(i))
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plan = make(B.FP32_BULK)
                plan.compute(phi32, stream=stream)
                e1.record(stream)
                stats.append(plan.stats())
                plan.close()
                times.append(e0.elapsed_time(e1))
        csum = clocks.summary()
        # End to end from pinned host buffers: the inputs' host-to-device copies,
        # bldtt_setup_batch + bldtt_compute, and phi back to the host.
        hp = torch.from_numpy(pts).pin_memory()
        hq = torch.from_numpy(q).pin_memory()
        hphi = torch.empty(M, dtype=torch.float64).pin_memory()
        dpts = torch.empty_like(dt)
        dqq = torch.empty_like(dq)
        e2e_times = []
        for i in range(1 + max(1, min(3, args.steps))):
            flush.fill_(float(i))
            stream.synchronize()
            t0 = time.perf_counter()
            dpts.copy_(hp, non_blocking=True)
            dqq.copy_(hq, non_blocking=True)
            plan = B.Plan.batch(dpts, off, dpts, off, dqq, kernels, kappas, precision=B.FP32_BULK,
                                stream=stream, **kw)
            plan.compute(phi32, stream=stream)
            hphi.copy_(phi32, non_blocking=True)
            stream.synchronize()
            t1 = time.perf_counter()
            plan.close()
            if i > 0:
                e2e_times.append(t1 - t0)
        e2e = {"value": M / statistics.median(e2e_times), "unit": UNIT,
               "h2d_bytes_per_step": int(hp.numel() * 8 + hq.numel() * 8),
               "d2h_bytes_per_step": int(M * 8), "seconds": statistics.median(e2e_times)}
    torch.cuda.synchronize()
    total_ms = sum(times)
    total_ms = max_over_ranks(total_ms, dist)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    st = stats[-1]
    value = job_rate(M, args.steps, world, total_ms)
    evals = sum(st["interactions"])
    ms_int = statistics.mean(s["ms_interact"] for s in stats)
    nyuk = sum(1 for k in kernels if k == B.YUKAWA)
    flops_per = (20.0 * (len(kernels) - nyuk) + 28.0 * nyuk) / len(kernels)
    props = torch.cuda.get_device_properties(local)
    peak = props.multi_processor_count * 128 * 2 * measured_peaks().get("sm_max_mhz", 2070.0) / 1e6
    achieved = flops_per * evals / (ms_int / 1000.0) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": (f"batched_512: {len(probs)} problems, N log-uniform in [1E3, 1E5] "
                                f"({M} targets in all), even cube / odd sphere surface, normal(0,1) "
                                f"charges, Coulomb or Yukawa kappa~U[0.1,2] ({nyuk} Yukawa), "
                                f"n={kw['n']}, theta={kw['theta']}, leaves {kw['N0']}, FP32 bulk; "
                                f"one plan; one persistent interaction launch drains the Coulomb and "
                                f"Yukawa work items together"),
                   "problems": len(probs), "M": M, "l2": "flushed between timed steps (256 MiB write)"},
        "rel_l2_vs_fp64": rel_l2, "worst_problem_rel_l2_vs_fp64": worst, "accuracy_ok": worst <= 1e-6,
        "phases_ms": {"tree": st["ms_tree"], "lists": st["ms_lists"], "upward": st["ms_upward"],
                      "interact": st["ms_interact"], "downward": st["ms_downward"],
                      "compute": st["ms_compute"]},
        "graph": {"autotuned_layout": layout, "ms_per_replay": statistics.median(graph_ms),
                  "targets_per_s": M / (statistics.median(graph_ms) / 1000.0)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_interact<FP32,mixed>",
                     "flops_per_launch": flops_per * evals, "ms_per_launch": ms_int},
        "gpu_launches": sum(s["launches_setup"] + s["launches_compute"] for s in stats),
        "fp64_plain": {"ms_compute": st64["ms_compute"]},
        "e2e": e2e, "clocks": csum, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_gpu_learned(args):
    """1E8 uniform points, Coulomb, leaves 2000, FP32 bulk: the learned pair
    selector (degrees 3..8, trained on the GPU on smaller problems with their
    own seeds, per-pair budget calibrated for 1e-6) against the fixed rule
    n=8, theta=0.7.  A step is setup + compute; errors are against the FP64
    direct sum on 1E4 sampled targets.  `value` is the learned path's rate."""
    import numpy as np
    import torch

    from paper_2012_06925_gb300 import binding as B
    from paper_2012_06925_gb300 import build as builder
    from paper_2012_06925_gb300 import selector as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    builder.build()
    B.load_library()
    t_train = time.perf_counter()
    sel, report = S.train_selector(budget=1e-6, epochs=200, seed=0)
    t_train = time.perf_counter() - t_train

    cfg, tgt, src, q, kw = workload(args.workload)
    M = tgt.shape[1]
    dt = torch.from_numpy(tgt).cuda()
    dq = torch.from_numpy(q).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    phi = torch.empty(M, dtype=torch.float64, device="cuda")
    base = dict(theta=kw["theta"], N0=kw["N0"], M0=kw["M0"], precision=B.FP32_BULK, stream=stream)

    def step(which):
        if which == "learned":
            plan = B.Plan.learned(dt, dt, dq, sel, **base)
        else:
            plan = B.Plan(dt, dt, dq, kernel=kw["kernel"], kappa=kw["kappa"], n=kw["n"], **base)
        plan.compute(phi, stream=stream)
        return plan

    idx = np.random.default_rng(77).choice(M, size=10_000, replace=False)
    idx.sort()
    errors = {}
    for which in ("fixed", "learned"):
        plan = step(which)
        plan.check_error()
        plan.close()
        errors[which] = S.sampled_error(tgt, q, phi.cpu().numpy(), idx)

    def timed(which):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            step(which).close()
        torch.cuda.synchronize()
        times, sts = [], []
        with ClockSampler(local) as clocks:
            for i in range(args.steps):
                flush.fill_(float(i))
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plan = step(which)
                e1.record(stream)
                sts.append(plan.stats())
                plan.close()
                times.append(e0.elapsed_time(e1))
        return sum(times), sts, clocks.summary()

    if dist is not None:
        dist.barrier()
    total_ms, sts, csum = timed("learned")
    total_ms = max_over_ranks(total_ms, dist)
    fixed_ms, fsts, _ = timed("fixed")
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    st, fst = sts[-1], fsts[-1]
    value = job_rate(M, args.steps, world, total_ms)
    ms_interact = statistics.mean(s["ms_interact"] for s in sts)
    flops = 20.0 * sum(st["interactions"])
    achieved = flops / (ms_interact / 1000.0) / 1e12
    props = torch.cuda.get_device_properties(local)
    sm_max = measured_peaks().get("sm_max_mhz", 2070.0)
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12

    # End to end through the public API: pinned host inputs in, potentials out.
    ht = torch.from_numpy(tgt).pin_memory()
    hq = torch.from_numpy(q).pin_memory()
    hphi = torch.empty(M, dtype=torch.float64).pin_memory()
    e2e_times = []
    for i in range(2):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dt2 = ht.cuda(non_blocking=True)
        dq2 = hq.cuda(non_blocking=True)
        plan = B.Plan.learned(dt2, dt2, dq2, sel, **base)
        plan.compute(phi, stream=stream)
        hphi.copy_(phi, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        plan.close()
        del dt2, dq2
    e2e = {"value": M / min(e2e_times), "unit": UNIT, "h2d_bytes_per_step": int(M * 32),
           "d2h_bytes_per_step": int(M * 8), "seconds": min(e2e_times)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(config_dict(cfg), workload=(
            "uniform_n1e8: 1E8 uniform in [-1,1]^3, targets=sources, charges U[-1,1], Coulomb, "
            "leaves 2000, FP32 bulk; learned selector (degrees 3..8, 6 features, 3x64 hidden, "
            "bf16) vs fixed n=8 theta=0.7; errors vs FP64 direct on 1E4 sampled targets")),
        "rel_l2_vs_fp64_direct": errors["learned"], "accuracy_ok": errors["learned"] <= 1e-6,
        "fixed_rule": {"value": M * args.steps / (fixed_ms / 1000.0), "unit": UNIT,
                       "ms_per_step": fixed_ms / args.steps,
                       "rel_l2_vs_fp64_direct": errors["fixed"],
                       "interactions": sum(fst["interactions"]),
                       "phases_ms": {k: fst["ms_" + k] for k in ("tree", "lists", "upward", "interact",
                                                                  "downward", "compute")}},
        "speedup_vs_fixed_rule": fixed_ms / total_ms,
        "selector": {"train_seconds": t_train, "pairs": report["pairs"], "loss": report["loss"],
                     "log10_pair_budget": report["log_eps"], "separation_cap": report["sep_cap"],
                     "degrees": list(sel.degrees)},
        "phases_ms": {k: st["ms_" + k] for k in ("tree", "lists", "upward", "interact", "downward",
                                                  "compute")},
        "interactions": {"PP": st["interactions"][0], "PC": st["interactions"][1],
                         "CP": st["interactions"][2], "CC": st["interactions"][3]},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "k_interact<FP32,Coulomb> (multi-degree)", "flops_per_launch": flops,
                     "ms_per_launch": ms_interact},
        "e2e": e2e, "gpu_launches": sum(s["launches_setup"] + s["launches_compute"] for s in sts),
        "clocks": csum, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched_512":
        return run_gpu_batched(args)
    if args.workload == "uniform_n1e8":
        return run_gpu_learned(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
