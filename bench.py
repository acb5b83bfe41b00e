#!/usr/bin/env python
"""Benchmark of one VMC + stochastic-reconfiguration step (the whole hot path).

Workload (default): 24 x 24 periodic Heisenberg antiferromagnet with the
Marshall sign folded in, real RBM alpha = 8 (M = 4608, Np = 2 659 392),
spin-exchange Metropolis at S_z = 0 with 8192 chains x 8 samples (Ns =
65536), eps = 0.01, lr = 0.01, SR solved by conjugate gradients on the
on-the-fly QGT (relative residual 1e-6 in NK_MIXED, 1e-10 in NK_F64).  A step
= sampling (8 sweeps per chain), local energies, statistics, force, SR solve
and update, all through nk_sr_step.  The same step on the FP64 GPU path
(fewer steps) and the other workloads are added to the line: the 10 x 10
Heisenberg (sample-space Cholesky), its symmetric RBM, the 20 x 20 Ising
(CG), J1-J2 on 10 x 10 and the 16-site Ising chain; then the t-VMC leg and
the serving stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|f64]
    python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Multi-GPU runs (torchrun) are independent replicas: the VMC step has no
data-parallel exchange on one GPU per box, so every rank runs its own chains
and the line reports the units all ranks processed over the slowest rank's
time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "VMC samples·sweeps/s & SR steps/s, mixed vs FP64 on 1 GB300; serve p50/p99"
FP64_PEAK_TFLOPS = 1.25     # nominal GB300 FP64 rate (CUDA cores)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x FMA x max clock


def measured_peaks():
    """Measured peaks of this GPU model from MEASURED_PEAKS.json (HBM copy
    GB/s, cuBLAS bf16 TF/s burst and sustained), else fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "of measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "of fallback"


# CG stopping rule per precision: relative residual 1e-10 on the FP64 path,
# 1e-6 on the mixed path (whose 3-slice FP16 QGT products carry about 2^-33)
CG_TOL = {"f64": 1e-10, "mixed": 1e-6}
# chains of the oracle's bounded sample per workload (about 10-30 s of one
# host thread per SR step; the default is used for the others)
ORACLE_CHAINS = {"heis2d_24x24": 4, "tfim2d_20x20": 16, "heis2d_10x10": 128}
ORACLE_CHAINS_DEFAULT = 64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "f64"])
    ap.add_argument("--workload", default="heis2d_24x24",
                    help="workload name, optionally with @rule to replace its sampler rule "
                         "(e.g. heis2d_10x10@hamiltonian)")
    ap.add_argument("--extra", default="heis2d_10x10,heis2d_10x10_symm,tfim2d_20x20,j1j2_10x10,tfim1d_n16",
                    help="comma-separated workloads timed after the headline (mixed path, same steps); none: no others")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the other-precision timing")
    ap.add_argument("--compare-steps", type=int, default=2,
                    help="timed steps of the other-precision arm (after one warm-up step)")
    ap.add_argument("--chains", type=int, default=0,
                    help="override the workload's chain count (a smaller case of the same kernels, for profilers)")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--tdvp", default="tdvp_tfim1d_l20",
                    help="t-VMC workload added to the line (none: skip)")
    ap.add_argument("--serve", type=int, default=512,
                    help="requests of the serving run added to the line (0: none)")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    return ap.parse_args()


def workload(name):
    from paper_2112_10526_gb300 import inputs as I
    base, _, rule = name.partition("@")
    w = dict(I.WORKLOADS[base])
    if rule:
        assert rule in ("local", "exchange", "hamiltonian"), rule
        w["rule"] = rule
    w["name"] = name
    w["ham"] = w["ham"]()
    if "symm" in w:
        w["perms"] = getattr(I, w["symm"])(int(round(w["N"] ** 0.5))) if w["symm"] == "translations_square" \
            else getattr(I, w["symm"])(w["N"])
        w["M"] = w["alpha"] * w["perms"].shape[0]  # expanded hidden units
        w["Np"] = 1 + w["alpha"] + w["alpha"] * w["N"]
    else:
        w["M"] = w["alpha"] * w["N"]
        w["Np"] = w["N"] + w["M"] + w["M"] * w["N"]
    return w


# ----------------------------------------------------------- CPU oracle ----

def oracle_chains(name):
    return ORACLE_CHAINS.get(name.partition("@")[0], ORACLE_CHAINS_DEFAULT)


def oracle_sample(name, chains, steps):
    """Time the oracle's SR step on `chains` chains of the workload, `steps`
    times (the first with the workload's discarded sweeps, untimed when more
    than one step is asked for).  Runs in a fresh process; the thread count
    comes from OMP_NUM_THREADS / OPENBLAS_NUM_THREADS."""
    import numpy as np
    import oracle
    from paper_2112_10526_gb300 import inputs as I
    w = workload(name)
    N, M = w["N"], w["M"]
    p = I.rbm_params(N, M, w["seed"])
    s = oracle.chain_init(N, chains, w["rule"], w["seed"], 0)
    times = []
    sweep0 = 0
    solver = "cg" if w["solver"] == "cg" else "cholesky"
    for k in range(steps):
        nd = w["discard"] if k == 0 else 0
        t0 = time.perf_counter()
        r = oracle.sr_step(p, N, M, w["ham"], w["rule"], s, sweep0, nd, w["per_chain"], w["seed"], 0,
                           diag_shift=w["diag_shift"], lr=w["lr"], solver=solver, cg_tol=CG_TOL["f64"],
                           cg_maxiter=1000)
        times.append(time.perf_counter() - t0)
        p, s = r["params"], r["state"]
        sweep0 += nd + w["per_chain"]
    return {"times": times, "energy": float(r["stats"]["mean"]), "cg_iters": int(r["cg_iters"]),
            "solver": solver}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_subprocess(name, chains, steps, threads):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample",
                          f"{name}:{chains}:{steps}"], env=env, capture_output=True, text=True,
                         check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_line_fields(name, chains, res, threads):
    """SR steps/s of the whole workload from the oracle's steps on `chains`
    chains (the work is per chain and per sample: linear extrapolation)."""
    w = workload(name)
    scale = w["chains"] / chains
    times = res["times"][1:] if len(res["times"]) > 1 else res["times"]
    t = statistics.median(times)
    value = 1.0 / (t * scale)
    return value, {
        "value": value, "unit": "SR steps/s", "cores": threads, "kind": "oracle",
        "sample": (f"{chains} of {w['chains']} chains x {w['per_chain']} samples, oracle {res['solver']} "
                   f"solver (CG: x0 = 0, tol {CG_TOL['f64']:g}), {threads} host thread(s); median of "
                   f"{len(times)} step(s) after the discard step, extrapolated linearly in the number of "
                   f"samples ({t:.2f} s per sampled step)"),
    }


def cpu_baseline(name):
    """The oracle timed on all host cores (the reported baseline) and on one
    thread, each on the bounded sample of the workload."""
    chains = oracle_chains(name)
    n = host_cores()
    wide = max(chains, min(n, workload(name)["chains"]))  # a chain per thread at least
    all_v, all_f = oracle_line_fields(name, wide, run_oracle_subprocess(name, wide, 2, n), n)
    one_v, one_f = oracle_line_fields(name, chains, run_oracle_subprocess(name, chains, 2, 1), 1)
    all_f["nproc"] = n
    all_f["single_thread"] = {"value": one_v, "unit": "SR steps/s", "cores": 1}
    return all_f


# --------------------------------------------------------------- clocks ----

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# ------------------------------------------------------------- our path ----

def setup(w, precision, rank, dev):
    import torch
    from paper_2112_10526_gb300 import inputs as I
    from paper_2112_10526_gb300 import nk
    N, M, C = w["N"], w["M"], w["chains"]
    st = {"N": N, "M": M, "C": C, "ns": w["per_chain"]}
    if "symm" in w:
        st["symm"] = (w["alpha"], torch.from_numpy(w["perms"].astype("int32")).to(dev))
        st["params"] = torch.from_numpy(I.symm_params(N, w["alpha"], w["seed"])).to(dev)
    else:
        st["params"] = torch.from_numpy(I.rbm_params(N, M, w["seed"])).to(dev)
    st["edges"] = torch.from_numpy(w["ham"]["edges"]).to(dev)
    st["ham"] = nk.make_ham(w["ham"]["kind"], w["ham"]["J"], w["ham"].get("h", 0.0),
                            w["ham"].get("marshall", False), st["edges"], w["ham"].get("J2", 0.0),
                            w["ham"].get("n_edges2", 0))
    st["s"] = torch.empty((C, N), dtype=torch.int8, device=dev)
    st["ctx"] = nk.Ctx(dev.index)
    nk.nk_chains_init(st["ctx"], N, C, w["rule"], w["seed"], rank, st["s"])
    st["chains"] = nk.make_chains(st["s"])
    st["cfg"] = nk.make_cfg(w["rule"], precision, w["solver"], w["discard"], w["per_chain"],
                            w["diag_shift"], w["lr"], w["seed"], stream_id=rank, cg_tol=CG_TOL[precision],
                            cg_maxiter=1000)
    st["stats"] = torch.empty(nk.SR_STATS_DOUBLES, dtype=torch.float64, device=dev)
    return st


def step(st, first=False):
    from paper_2112_10526_gb300 import nk
    st["cfg"].n_discard = st["cfg"].n_discard if first else 0
    if "symm" in st:
        alpha, perms = st["symm"]
        nk.nk_symm_sr_step(st["ctx"], st["params"], st["N"], alpha, perms, st["ham"], st["chains"], st["cfg"],
                           st["stats"])
        return
    nk.nk_sr_step(st["ctx"], st["params"], st["N"], st["M"], st["ham"], st["chains"], st["cfg"],
                  st["stats"])


def lattice_text(N):
    L = int(round(N ** 0.5))
    return f"{L}x{L} periodic square" if L * L == N else f"{N}-site periodic chain"


def ham_text(ham):
    if ham.get("n_edges2", 0):
        return f"{ham['kind']} J1-J2 (J1={ham['J']}, J2={ham['J2']}, exchange over both edge classes)"
    return ham["kind"]


def l2_text(solver, Ns, M, Np):
    """Which per-step array outgrows the 129 MB L2 between timed steps."""
    if solver == "cholesky_samplespace":
        what, nbytes = "Ns x Ns FP64 Gram", Ns * Ns * 8
    elif solver == "cholesky":
        what, nbytes = "Np x Np FP64 QGT", Np * Np * 8
    else:
        what, nbytes = "Ns x M FP64 tanh(theta), read per CG product", Ns * M * 8
    side = "larger" if nbytes > 129e6 else "SMALLER"
    return f"working set {side} than L2 ({what} = {nbytes / 2**20:.0f} MiB per step)"


def replica_value(world, K, ms_max):
    """Whole-job SR steps/s of `world` independent replicas that each ran K
    steps, from the slowest rank's time (ms): weak scaling."""
    return world * K / (ms_max / 1e3)


def barrier(world):
    import torch.distributed as dist
    if world > 1:
        dist.barrier()


def max_over_ranks(x, world, dev):
    import torch
    import torch.distributed as dist
    if world == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed_steps(st, K, world, dev, prof=False):
    """K steps bracketed by a barrier and a synchronize on both sides, timed
    with CUDA events on the launching stream.  With prof, every tracked
    kernel class is also timed by the library's own events (on the streams
    its kernels run on) and its algorithmic and executed work added up."""
    import torch
    from paper_2112_10526_gb300 import nk
    stream = torch.cuda.current_stream()
    barrier(world)
    torch.cuda.synchronize()
    if prof:
        nk.nk_prof_enable(True)
    l0 = nk.nk_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        step(st)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = nk.nk_launch_count() - l0
    ms = e0.elapsed_time(e1)
    prof_out = None
    if prof:
        prof_out = {c: nk.nk_prof_read(c) + (nk.nk_prof_read_executed(c),) for c in nk.PROF_CLASSES}
        nk.nk_prof_enable(False)
    return max_over_ranks(ms, world, dev), launches, prof_out


def e2e_steps(st, K, dev):
    """Each step: pinned host -> device copy of the step's inputs (parameters
    and chain states), nk_sr_step, device -> host read of the result
    (updated parameters and the step statistics)."""
    import torch
    from paper_2112_10526_gb300 import nk
    h_params = st["params"].cpu().pin_memory()
    h_s = st["s"].cpu().pin_memory()
    h_out = torch.empty_like(h_params).pin_memory()
    h_stats = torch.empty(nk.SR_STATS_DOUBLES, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        st["params"].copy_(h_params, non_blocking=True)
        st["s"].copy_(h_s, non_blocking=True)
        step(st)
        h_out.copy_(st["params"], non_blocking=True)
        h_stats.copy_(st["stats"], non_blocking=True)
        torch.cuda.current_stream().synchronize()
        h_params.copy_(h_out)
    dt = time.perf_counter() - t0
    bi = h_params.numel() * 8 + h_s.numel()
    bo = h_out.numel() * 8 + 8 * 8
    return dt, bi, bo


# DRAM bytes (read + write) per launch of the dominant kernels, from one ncu
# capture each (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the
# sha256 of the kernel's own source section so that a changed kernel reports
# no stale figure.
# k_ozaki_gemm: per 128 x 32 output tile with 7 slices (the 8064 x 8064
# lower update of the 10 x 10 workload: 472.76 MB over 8064 tiles).
OZAKI_TRAFFIC = {"bytes_per_tile": 59062.3, "source_sha256_prefix": "393611d8bf30c3e9"}
OZAKI_TILE_FLOPS = 28 * 4 * 2.0 * 128 * 32 * 16  # executed BF16 flops per tile (7 slices)
# k_tc4 (the CG's J v and J^T g products): bytes per launch captured on the
# 24 x 24 workload at 1024 chains (Ns = 8192): J v 331.97 MB read + 3.59 MB
# written, J^T g 243.31 + 27.24 MB.  Both read their operands once, which
# grow with Ns (the tanh(theta) pairs, the +-1 operand, the (T' o g')^T
# digits), so a launch at Ns samples moves about Ns / 8192 times as much.
TC4_TRAFFIC = {"ns": 8192, "jv": 335554304, "jtg": 270545664, "source_sha256_prefix": "5e16dbda6876423f"}


def _section_hash(fname, start, end):
    import hashlib
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2112_10526_gb300", "csrc")
    try:
        s = open(os.path.join(here, fname)).read()
        return hashlib.sha256(s[s.index(start):s.index(end)].encode()).hexdigest()
    except (OSError, ValueError):
        return ""


def ozaki_source_hash():
    return _section_hash("k_tc.cu", "// ------------------------------------------------------------- the GEMM ---",
                         "// ------------------------------------------------- Cholesky building blocks ---")


def tc4_source_hash():
    return _section_hash("k_sgemm.cu", "// ------------------------------ J v and J^T g: persistent, 3 FP16 slices ---",
                         "// ------------------------------------------------------- operand staging ---")


TENSOR_CLASSES = ("chol_update", "gram", "jvp_vjp")


def class_roofline(cls, ms, launches, work, executed, precision):
    """One kernel class against the roofline that bounds it.  `work` is the
    method's algorithmic work (ratio terms for the sweep and the local
    energies, FP64-operation flops for the products and factorisations);
    `executed` what the hardware ran (BF16 slice-product flops of the
    tensor-core paths)."""
    peaks, src = measured_peaks()
    secs = ms / 1e3
    out = {"kernel_class": cls, "launches": launches, "avg_launch_ms": ms / launches}
    if cls in ("sweep", "eloc"):
        # one FMA and one multiply per ratio term
        out.update(bound="alu", unit="TFLOP/s", achieved=2.0 * work / secs / 1e12,
                   algorithmic_work="2 flops per ratio term")
        if precision == "f64":
            out.update(peak=FP64_PEAK_TFLOPS, peak_source="FP64 pipe, nominal 1.25 TFLOP/s (of nominal)")
        else:
            out.update(peak=FP32_PEAK_TFLOPS,
                       peak_source="FP32 lanes: 152 SMs x 128 x 2 x 2.07 GHz (of nominal)")
    elif cls in TENSOR_CLASSES and precision == "mixed":
        out.update(bound="tensor", unit="TFLOP/s", achieved=work / secs / 1e12,
                   peak=peaks["bf16_tflops_sustained"],
                   peak_source=f"bf16 dense, sustained ({src}); the products run as BF16 / FP16 integer-slice "
                               f"products (FP16 at the BF16 rate)",
                   algorithmic_work="flops of the FP64 operation",
                   executed_tflops=executed / secs / 1e12,
                   executed_frac=executed / secs / 1e12 / peaks["bf16_tflops_sustained"])
    elif cls == "trsv":
        # two solves read the lower factor once each: n^2 / 2 x 8 bytes per solve, work = 2 n^2
        out.update(bound="hbm", unit="GB/s", achieved=(work / 2.0) * 8.0 / secs / 1e9, peak=peaks["hbm_gbs"],
                   peak_source=f"HBM copy ({src})", algorithmic_work="the lower factor read once per solve")
    else:
        out.update(bound="alu", unit="TFLOP/s", achieved=work / secs / 1e12, peak=FP64_PEAK_TFLOPS,
                   peak_source="FP64 pipe, nominal 1.25 TFLOP/s (of nominal; no measured FP64 peak)",
                   algorithmic_work="FP64 flops")
    out["frac"] = out["achieved"] / out["peak"]
    return out


def roofline(prof, K, precision, ns=None):
    """The dominant tracked kernel class by time, with its DRAM traffic per
    launch where a capture of the same kernel source exists (ns: the
    workload's samples, for the Jacobian products)."""
    cls = max(prof, key=lambda c: prof[c][0])
    ms, launches, work = prof[cls][:3]
    executed = prof[cls][3] if len(prof[cls]) > 3 else work
    if launches == 0 or ms <= 0:
        return None, cls
    rf = class_roofline(cls, ms, launches, work, executed, precision)
    traffic = None
    if cls == "chol_update" and precision == "mixed" and \
            ozaki_source_hash().startswith(OZAKI_TRAFFIC["source_sha256_prefix"]):
        # bytes per launch, like achieved: the class's tiles x the captured bytes per tile
        traffic = executed / OZAKI_TILE_FLOPS * OZAKI_TRAFFIC["bytes_per_tile"] / launches
    if cls == "jvp_vjp" and precision == "mixed" and ns and \
            tc4_source_hash().startswith(TC4_TRAFFIC["source_sha256_prefix"]):
        # the mean of a J v and a J^T g launch of k_tc4, scaled to the workload's Ns
        traffic = 0.5 * (TC4_TRAFFIC["jv"] + TC4_TRAFFIC["jtg"]) * ns / TC4_TRAFFIC["ns"]
        rf["traffic_kernel"] = "k_tc4 (mean of J v and J^T g), captured at Ns = 8192 and scaled by Ns"
    rf["traffic"] = traffic
    rf["traffic_unit"] = "DRAM bytes per launch"
    return rf, cls


def rooflines_by_class(prof, step_ms, precision):
    """Every tracked kernel class per step against its roofline."""
    out = {}
    for cls, v in prof.items():
        ms, launches, work = v[:3]
        executed = v[3] if len(v) > 3 else work
        if launches == 0 or ms <= 0:
            continue
        r = class_roofline(cls, ms, launches, work, executed, precision)
        r.update(ms_per_step=ms, share_of_step=ms / step_ms)
        out[cls] = r
    return out


def measure(w, precision, K, warmup, rank, world, dev, prof=True, e2e=True):
    """Warm-up, a profiled timing (per-class events), the plain timing (the
    headline number) and the end-to-end timing of one workload."""
    from paper_2112_10526_gb300 import nk
    st = setup(w, precision, rank, dev)
    for i in range(warmup):
        step(st, first=(i == 0))
    import torch
    torch.cuda.synchronize()
    # The profiled, plain and end-to-end timings replay the same K steps: the
    # state after the warm-up (parameters, chains, sweep counter) is restored
    # before each, and the steps are deterministic, so the per-class split and
    # the CG iteration counts belong to the steps the headline times.
    snap = (st["params"].clone(), st["s"].clone(), st["chains"].sweeps_done)

    def restore():
        st["params"].copy_(snap[0])
        st["s"].copy_(snap[1])
        st["chains"].sweeps_done = snap[2]
        torch.cuda.synchronize()

    res = {}
    if prof:
        ms_p, _, pr = timed_steps(st, K, world, dev, prof=True)
        res["prof"], res["ms_prof"] = pr, ms_p
        restore()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    ms, launches, _ = timed_steps(st, K, world, dev, prof=False)
    res["clocks"] = clocks.stop()
    res["ms"], res["launches"] = ms, launches
    res["stats"] = nk.sr_stats_dict(st["stats"])
    if e2e:
        restore()
        dt, bi, bo = e2e_steps(st, K, dev)
        res["e2e"] = (max_over_ranks(dt, world, dev), bi, bo)
    st["ctx"].close()
    return res


def workload_config(w, precision, world):
    Ns = w["chains"] * w["per_chain"]
    Np = w["Np"]
    cfg = {"workload": w["name"], "lattice": lattice_text(w["N"]), "hamiltonian": ham_text(w["ham"]),
           "model": (f"symmetric RBM, alpha = {w['alpha']} over {w['perms'].shape[0]} translations"
                     if "symm" in w else f"RBM, alpha = {w['alpha']}"),
           "N": w["N"], "M": w["M"], "Np": Np, "chains": w["chains"], "samples_per_chain": w["per_chain"],
           "Ns": Ns, "rule": w["rule"], "solver": w["solver"], "precision": precision,
           "diag_shift": w["diag_shift"], "lr": w["lr"], "parallelism": f"replicas x{world}",
           "l2": l2_text(w["solver"], Ns, w["M"], Np)}
    if w["solver"] == "cg":
        cfg["cg_tol"] = CG_TOL[precision]
    return cfg


def run_ours(args, rank, world):
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.workload)
    if args.chains > 0:
        w["chains"] = args.chains
        w["name"] += f"@chains={args.chains}"
    K = args.steps
    r = measure(w, args.precision, K, args.warmup, rank, world, dev)
    ms_plain, prof = r["ms"], r["prof"]
    value = replica_value(world, K, ms_plain)
    stats = r["stats"]
    prof_step = {c: (v[0] / K, v[1] / K, v[2] / K, v[3] / K) for c, v in prof.items()}
    Ns = w["chains"] * w["per_chain"]
    rf, dom = roofline(prof, K, args.precision, ns=Ns)
    if rf is not None:
        rf["share_of_step"] = prof[dom][0] / r["ms_prof"]
    e2e_dt, bi, bo = r["e2e"]
    line = {
        "metric": METRIC, "value": value, "unit": "SR steps/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_plain / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "f64" else "f32+f64",
        "data": "synthetic (seeded RBM parameters N(0, 0.01^2), Philox chains)",
        "config": workload_config(w, args.precision, world),
        "samples_sweeps_per_s": world * K * Ns / (ms_plain / 1e3),
        "proposals_per_s": world * K * Ns * w["N"] / (ms_plain / 1e3),
        # local-energy evaluations per second of the E_loc kernels alone (CUDA events)
        "eloc_evals_per_s": (world * K * Ns / (prof["eloc"][0] / 1e3)) if prof.get("eloc", (0,))[0] > 0 else None,
        "energy": stats["energy"], "energy_error": stats["error"], "acceptance": stats["acceptance"],
        "cg_iters": stats["cg_iters"],
        "roofline": rf,
        "rooflines_by_class": rooflines_by_class(prof_step, r["ms_prof"] / K, args.precision),
        "kernel_ms_per_step": {c: prof[c][0] / K for c in prof if prof[c][1] > 0},
        "e2e": {"value": world * K / e2e_dt, "unit": "SR steps/s", "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo},
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
    }
    if not args.no_compare and world == 1:
        other = "f64" if args.precision == "mixed" else "mixed"
        Kc = max(1, args.compare_steps)
        r2 = measure(w, other, Kc, 1, rank, world, dev, prof=False, e2e=False)
        s2 = r2["stats"]
        line[f"{other}_path"] = {"value": Kc / (r2["ms"] / 1e3), "unit": "SR steps/s",
                                 "ms_per_step": r2["ms"] / Kc, "steps": Kc, "warmup": 1,
                                 "energy": s2["energy"], "energy_error": s2["error"],
                                 "cg_iters": s2["cg_iters"], "clocks": r2["clocks"],
                                 "config": workload_config(w, other, world)}
        # the energies of both precisions after the same 1 + Kc steps from the
        # same parameters, chains and Philox streams
        r3 = measure(w, args.precision, Kc, 1, rank, world, dev, prof=False, e2e=False)
        s3 = r3["stats"]
        line["energy_after_equal_steps"] = {
            "steps": 1 + Kc, args.precision: {"energy": s3["energy"], "error": s3["error"]},
            other: {"energy": s2["energy"], "error": s2["error"]},
            "difference_in_combined_errors": abs(s3["energy"] - s2["energy"]) /
            max(1e-300, (s3["error"] ** 2 + s2["error"] ** 2) ** 0.5)}
    extra = {}
    for name in [x for x in args.extra.split(",") if x and x != "none"] if world == 1 else []:
        we = workload(name)
        re_ = measure(we, args.precision, K, args.warmup, rank, world, dev)
        Ke = K
        dom_rf, _ = roofline(re_["prof"], Ke, args.precision, ns=we["chains"] * we["per_chain"])
        extra[name] = {"value": Ke / (re_["ms"] / 1e3), "unit": "SR steps/s", "ms_per_step": re_["ms"] / Ke,
                       "e2e": {"value": Ke / re_["e2e"][0], "unit": "SR steps/s",
                               "h2d_bytes_per_step": re_["e2e"][1], "d2h_bytes_per_step": re_["e2e"][2]},
                       "energy": re_["stats"]["energy"], "energy_error": re_["stats"]["error"],
                       "kernel_ms_per_step": {c: v[0] / Ke for c, v in re_["prof"].items() if v[1] > 0},
                       "roofline": dom_rf, "config": workload_config(we, args.precision, world)}
    if extra:
        line["other_workloads"] = extra
    return line


# ------------------------------------------------------------------ t-VMC ----

def run_tdvp(name, K, warmup, dev):
    """Time evolution of the complex RBM: K t-VMC steps (nk_tdvp_step, two
    slopes each for Heun) after `warmup` steps; CUDA events on the stream."""
    import numpy as np
    import torch
    from paper_2112_10526_gb300 import inputs as I
    from paper_2112_10526_gb300 import nk
    w = dict(I.TDVP_WORKLOADS[name])
    N, M, C = w["N"], w["alpha"] * w["N"], w["chains"]
    ham = w["ham"]()
    params = torch.from_numpy(I.complex_rbm_params(N, M, w["seed"], w["sigma"])).to(dev)
    edges = torch.from_numpy(ham["edges"]).to(dev)
    h = nk.make_ham(ham["kind"], ham["J"], ham.get("h", 0.0), ham.get("marshall", False), edges)
    s = torch.from_numpy(I.random_configs(C, N, w["seed"])).to(dev)
    ch = nk.make_chains(s)
    cfg = nk.make_tdvp_cfg(w["rule"], w["integrator"], w["real_time"], w["solver"], w["discard"], w["per_chain"],
                           w["dt"], w["diag_shift"], w["seed"], rcond=w["rcond"])
    stats = torch.empty(4, dtype=torch.float64, device=dev)
    with nk.Ctx(dev.index) as ctx:
        for i in range(max(1, warmup)):
            nk.nk_tdvp_step(ctx, params, N, M, h, ch, cfg, stats)
            cfg.n_discard = 0
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            nk.nk_tdvp_step(ctx, params, N, M, h, ch, cfg, stats)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    st = stats.cpu().numpy()
    Ns = C * w["per_chain"]
    return {"value": K / (ms / 1e3), "unit": "t-VMC steps/s", "ms_per_step": ms / K, "steps": K,
            "energy": complex(st[0], st[1]).real, "energy_imag": float(st[1]), "energy_error": float(st[3]),
            "config": {"workload": name, "lattice": lattice_text(N), "hamiltonian": "tfim (h = 1 quench)",
                       "model": "complex RBM, alpha = 1", "N": N, "M": M, "Np_complex": N + M + M * N,
                       "chains": C, "samples_per_chain": w["per_chain"], "Ns": Ns, "integrator": w["integrator"],
                       "dt": w["dt"], "time": "real", "solver": f"pseudo-inverse (rcond {w['rcond']:g}), "
                       f"Jacobi on the {2 * (N + M + M * N)}-dim real embedding", "precision": "f64"}}


# ---------------------------------------------------------------- serving ----

def run_serve(n_requests, slots, budget_gb, device=0):
    """Serving workload: closed-loop capacity first (all requests queued at
    once), then Poisson arrivals at 0.8 x that rate; latency = submit ->
    completion as the server records it."""
    import threading
    import numpy as np
    from paper_2112_10526_gb300 import inputs as I
    from paper_2112_10526_gb300 import nk
    specs = I.serve_requests(n_requests, seed=4)

    def make(spec):
        cfg = nk.make_cfg(spec["rule"], "mixed", spec["solver"], 8, spec["per_chain"], 0.01, 0.01, spec["seed"],
                          stream_id=spec["index"], cg_tol=1e-8, cg_maxiter=200)
        p = I.rbm_params(spec["N"], spec["M"], spec["seed"])
        return nk.make_request("sr_step", spec["N"], spec["M"], p, spec["ham"], spec["chains"], cfg)

    reqs = [make(sp) for sp in specs]
    budget = int(budget_gb * (1 << 30))
    # closed loop
    with nk.Server(device, budget, slots) as srv:
        t0 = time.perf_counter()
        ids = [srv.submit(r) for r in reqs]
        res = [srv.wait(i) for i in ids]
        closed = time.perf_counter() - t0
        st_closed = srv.stats()
    capacity = n_requests / closed
    rate = 0.8 * capacity
    arrivals = I.poisson_arrivals(n_requests, rate, seed=4)
    with nk.Server(device, budget, slots) as srv:
        ids = [None] * n_requests
        t0 = time.perf_counter()

        def feeder():
            for k, at in enumerate(arrivals):
                delay = at - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                ids[k] = srv.submit(reqs[k])

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        res_open = [srv.wait(i) for i in ids]
        makespan = time.perf_counter() - t0
        st_open = srv.stats()
    lat = np.array([r["latency_ms"] for r in res_open])
    failed = sum(1 for r in res_open if r["status"] != 0)
    codes = {}
    for r in list(res) + list(res_open):
        if r["status"] != 0:
            codes[str(r["status"])] = codes.get(str(r["status"]), 0) + 1
    return {"requests": n_requests, "slots": slots, "hbm_budget_gb": budget_gb,
            "closed_loop_req_per_s": capacity, "arrival_rate_req_per_s": rate,
            "req_per_s": n_requests / makespan, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "failed": failed + st_closed["failed"], "failure_codes": codes,
            "failures": [(r["status"], r["message"]) for r in list(res) + list(res_open) if r["status"] != 0][:4],
            "mix": "Ising chains N in {16..256}, Heisenberg L in {4..16}, alpha in {1,2,4}, "
                   "1024 chains x U{1..16} samples, NK_MIXED, Cholesky if Np <= 4096 else CG (<= 200 it)"}


def main():
    args = parse()
    if args.oracle_sample:
        name, chains, steps = args.oracle_sample.split(":")
        print(json.dumps(oracle_sample(name, int(chains), int(steps))))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return
        n = host_cores()
        chains = max(oracle_chains(args.workload), min(n, workload(args.workload)["chains"]))
        res = run_oracle_subprocess(args.workload, chains, args.steps + args.warmup, n)
        res["times"] = res["times"][args.warmup:] or res["times"]
        value, cpu = oracle_line_fields(args.workload, chains, {**res, "times": [0.0] + res["times"]}, n)
        cpu["nproc"] = n
        w = workload(args.workload)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "SR steps/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(w, "f64", 1),
                "cpu_baseline": cpu,
                "e2e": {"value": value, "unit": "SR steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle runs in fresh processes before any CUDA work in this one
        cpu = cpu_baseline(args.workload)
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    line = run_ours(args, rank, world)
    line["cpu_baseline"] = cpu
    if args.tdvp and args.tdvp != "none" and world == 1:
        import torch
        line["tdvp"] = run_tdvp(args.tdvp, args.steps, args.warmup,
                                torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0"))))
    if args.serve > 0 and world == 1:
        line["serve"] = run_serve(args.serve, args.serve_slots, args.serve_budget_gb,
                                  int(os.environ.get("LOCAL_RANK", "0")))
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
