#!/usr/bin/env python3
"""Benchmark of the seed solver on GB300.

Metric: all-RHS time to solution at relative residual 1e-8 for the Wilson
workload -- an 8^4 lattice (n = 49152 complex unknowns), kappa = 0.155,
SU(3) links exp(0.3 i H) from seed 0, 12 unit point sources eta (site 0,
every spin and colour), normal equations A = D^H D with b^j = D^H eta^j
(Sec. 4).  One step = form B = D^H eta, seed solve of system 1 to 1e-12 with
reorthogonalization every 100 steps (Sec. 3), CG on systems 2..12 to 1e-8.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun each rank solves its own replica of the
workload (the path is single-GPU; N GPUs run N independent problems).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "all-RHS solve time at rel. residual 1e-8; matvec HBM GB/s vs GB300 peak"
WL = dict(dims=(8, 8, 8, 8), kappa=0.155, link_eps=0.3, link_seed=0, nrhs=12, m_max=3000, reorth_freq=100,
          reorth_passes=2, tol_seed=1e-12, tol_rest=1e-8)
WORKLOAD_NAME = "wilson-dirac 8^4 kappa=0.155 A=D^H D, 12 point sources, seed tol 1e-12 reorth/100, CG tol 1e-8"
# Wilson D per site: 1320 flops for the eight spin-projected hops (colour matrix times two
# half-spinors, reconstruction and accumulation; FMA = 2 flops), the usual count for this operator.
# The epilogue psi - kappa * sum adds 48 more, which the roofline reports separately.
FLOPS_PER_SITE_D = 1320
FLOPS_PER_SITE_D_EPILOGUE = 48
# FP64 instructions the kernel issues per site (each a full FMA slot whether it is an FMA, a multiply
# or an add): 4 directions x (84 + 96) for the fused hop pairs, 72 adds combining the four direction
# partials, 24 FMAs of psi - kappa * sum.  1320 counted flops over 2 x 816 slots: the kernel cannot
# exceed 0.809 of the unit-count peak.
FP64_INSTR_PER_SITE_D = 816
# FP64 peak from unit counts: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (the library's FMA-chain
# probe, seed_time_fma, measures it live next to the roofline)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
try:
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as _fh:
        MEASURED_PEAKS = json.load(_fh)
except (OSError, ValueError):
    MEASURED_PEAKS = {}
# DRAM bytes of one k_dslash launch (8^4, 11 columns) from the ncu capture of these sources of the
# kernel; reported only while the source is unchanged.
DSLASH_TRAFFIC = {"fa1e067f137fcf97": 11.207168e6 + 0.0, "6e70bd4a297626c1": 11.207424e6 + 0.0,
                 "ea8d71246ee34395": 11.207424e6 + 0.0}
# The same for k_dslash32_site<+1> (FP32, 16^3 x 32, 11 columns), from the ncu capture of its sources
DSLASH32_TRAFFIC = {"7a583b64681e7245": 189.553920e6 + 104.930304e6}
DSLASH32_TRAFFIC_DIMS = (16, 16, 16, 32)


def cg_branch_cols(nc, branches=3):
    """Columns per branch of the library's lockstep CG graphs (two or more columns per branch)."""
    nb = max(1, min(branches, nc // 2))
    start = [b * nc // nb for b in range(nb + 1)]
    return [start[b + 1] - start[b] for b in range(nb)]


def fp32_kernel_name(sites):
    """The FP32 hopping kernel the library runs on a lattice of this many sites."""
    return "k_dslash32_site" if sites >= 65536 else "k_dslash32"


def dslash_source_hash(fp32=False):
    """Hash of the hopping kernel's sources (the .cu and its device header)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("wilson32.cu" if fp32 else "wilson.cu", "wilson_device.cuh"):
        with open(os.path.join(ROOT, "paper_0810_0330_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dslash_traffic(fp32=False):
    return (DSLASH32_TRAFFIC if fp32 else DSLASH_TRAFFIC).get(dslash_source_hash(fp32))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 16^3 x 32 mixed-precision and FP64 solves reported under config.secondary")
    ap.add_argument("--kernel-only", action="store_true",
                    help="only time the dominant kernel (for profiler captures)")
    ap.add_argument("--once", action="store_true",
                    help="run the workload's step once and print its phase times, no bench line "
                         "(for launch-list captures)")
    ap.add_argument("--laplacian-once", action="store_true",
                    help="run the 64x64 Laplacian all-RHS solve once and print its phase times (for "
                         "launch-list captures)")
    ap.add_argument("--dims", default=None, help="lattice for --kernel-only, e.g. 16,16,16,16")
    ap.add_argument("--ncols", type=int, default=None, help="columns for --kernel-only")
    ap.add_argument("--reps", type=int, default=20, help="timed launches for --kernel-only")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="mixed: FP32 operator and Krylov vectors, FP64 scalars and reliable updates")
    ap.add_argument("--lattice", default=None,
                    help="lattice of the solve workload, e.g. 16,16,16,32 (default 8,8,8,8)")
    ap.add_argument("--sources", choices=["point", "z4"], default="point",
                    help="right-hand sides: 12 unit point sources at site 0, or 12 Z4 noise vectors (seed 0)")
    ap.add_argument("--csr-side", type=int, default=None,
                    help="--kernel-only on the 2-d Laplacian CSR of this side instead of the Wilson operator")
    ap.add_argument("--batched", action="store_true",
                    help="32 uneven shifted 2-d/3-d Laplacians (n 1e4..1e6, 4..16 RHS): sequential vs batched")
    ap.add_argument("--adjoint", action="store_true",
                    help="forward + backward of the differentiable solve: 16^4, kappa 0.150, 8 Gaussian b and t")
    ap.add_argument("--reorth-freq", type=int, default=None, help="reorthogonalization frequency for --adjoint")
    ap.add_argument("--reliable-delta", type=float, default=0.0,
                    help="mixed precision: reliable-update threshold (0: the library default, 0.001)")
    ap.add_argument("--sweep", action="store_true",
                    help="operator-apply bandwidth sweep (CSR Laplacian and Wilson D at growing sizes)")
    ap.add_argument("--sweep-max", type=int, default=3, help="sweep points per operator (1..4)")
    return ap.parse_args()


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


# A replica that dies or hangs must not leave the others waiting forever: the
# process group's timeout ends their next barrier or reduction with an error.
# It exceeds the longest healthy gap between two collectives (set-up, warm-up
# and the timed steps of one rank: a few minutes at most).
REPLICA_TIMEOUT_S = 600


def init_replicas(backend, device_id=None, timeout_s=REPLICA_TIMEOUT_S):
    import datetime
    import torch.distributed as dist
    kw = dict(timeout=datetime.timedelta(seconds=timeout_s))
    if device_id is not None:
        kw["device_id"] = device_id
    dist.init_process_group(backend, **kw)
    return dist


def replicas_barrier(dist, where):
    """Barrier of the replicas; raises (instead of hanging) when another rank
    has exited or stopped answering."""
    try:
        dist.barrier()
    except Exception as e:
        raise RuntimeError("replica barrier '%s' failed on rank %d: another rank has exited or stopped (%s)"
                           % (where, dist.get_rank(), e)) from e


def max_over_ranks(x, dist, dev):
    """The maximum of a per-rank time over all ranks (x itself without a
    process group).  Replicas run independent problems, so the job's time is
    that of its slowest rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, device_uuid=None):
        self.uuid = device_uuid
        self.proc = None

    def __enter__(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                self.rows.append(p)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on the whole workload
# ---------------------------------------------------------------------------
ARM_PARTS = {("0x41", "0xd4f"): "Arm Neoverse-V2", ("0x41", "0xd40"): "Arm Neoverse-V1",
             ("0x41", "0xd0c"): "Arm Neoverse-N1"}


def host_cpu():
    """(logical cores, CPU model) of this host (x86 'model name'; Arm implementer and part)."""
    model, impl, part = None, None, None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k = line.split(":")[0].strip().lower()
                val = line.split(":", 1)[1].strip() if ":" in line else ""
                if k in ("model name", "cpu model") and model is None:
                    model = val
                elif k == "cpu implementer" and impl is None:
                    impl = val
                elif k == "cpu part" and part is None:
                    part = val
    except OSError:
        pass
    if model is None and impl is not None:
        model = ARM_PARTS.get((impl.lower(), (part or "").lower()), "Arm implementer %s part %s" % (impl, part))
    if model is None:
        import platform
        model = platform.machine()
    return os.cpu_count() or 1, model


def oracle_full(threads=1):
    """The whole all-RHS solve by the oracle: B = D^H eta for the 12 sources, the
    seed solve of system 1, CG on all 11 seeded systems.  threads > 1 runs the
    oracle's OpenMP build (the same results bit for bit).  Returns
    (seconds, detail)."""
    import oracle
    from paper_0810_0330_gb300 import inputs as I
    used = oracle.set_threads(threads)
    dims, kappa = WL["dims"], WL["kappa"]
    U = I.random_su3_links(dims, WL["link_eps"], seed=WL["link_seed"])
    eta = I.point_sources(dims, WL["nrhs"])
    op = oracle.Operator.wilson(dims, kappa, U)
    t0 = time.perf_counter()
    B = np.stack([oracle.wilson_dslash(dims, kappa, 0, -1, U, eta[:, j]) for j in range(WL["nrhs"])], axis=1)
    r = oracle.seed_solve_all(op, B, m_max=WL["m_max"], reorth_freq=WL["reorth_freq"],
                              reorth_passes=WL["reorth_passes"], tol_seed=WL["tol_seed"], tol_rest=WL["tol_rest"])
    t1 = time.perf_counter()
    oracle.set_threads(1)
    ok = all(x["converged"] for x in r["rest"])
    return t1 - t0, dict(threads=used, seed_iters=r["seed"]["iters"], cg_iters=[x["iters"] for x in r["rest"]],
                         converged=ok)


def cpu_obj(total_s, d):
    cores, model = host_cpu()
    return {"value": round(total_s * 1e3, 3), "unit": "ms", "cores": d["threads"], "kind": "oracle",
            "host": {"logical_cores": cores, "cpu": model},
            "sample": "the whole workload, not a sample: the oracle (plain C, FP64, %s) forms B = D^H eta for "
                      "the 12 sources, runs the seed solve of system 1 (%d Lanczos steps) and CG on all 11 "
                      "seeded systems (%s iterations)" % (
                          "one thread" if d["threads"] == 1 else
                          "its OpenMP build on %d threads, results bit-identical to one thread" % d["threads"],
                          d["seed_iters"], d["cg_iters"])}


def cpu_baseline_obj():
    """One-thread oracle (as it stands) and the same source on every host core."""
    t1, d1 = oracle_full(1)
    out = cpu_obj(t1, d1)
    try:
        tn, dn = oracle_full(os.cpu_count() or 1)
        out["all_cores"] = cpu_obj(tn, dn)
    except Exception as e:   # no OpenMP toolchain on this host
        out["all_cores"] = {"unavailable": str(e)[:200]}
    return out


def run_reference(args):
    """The oracle as the reference arm: each step is the whole all-RHS solve of the
    workload on every host core (the OpenMP build of the oracle; results
    bit-identical to its one-thread build)."""
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    times = []
    detail = None
    for step in range(args.warmup + args.steps):
        t, d = oracle_full(threads)
        if step >= args.warmup:
            times.append(t)
            detail = d
    ms = statistics.mean(times) * 1e3
    out = {"metric": METRIC, "value": round(ms, 3), "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": workload_config(WL["dims"], "point", False, world),
           "impl_note": "the CPU oracle (the paper publishes no code), whole workload per step, all host cores",
           "cpu_baseline": cpu_obj(ms / 1e3, detail),
           "run": {"step_ms": [round(t * 1e3, 3) for t in times], "converged": detail["converged"]},
           "e2e": {"value": round(ms, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    out["cpu_baseline"]["value"] = out["value"]
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# operator-apply sweep: sizes below and above the 129 MB L2
# ---------------------------------------------------------------------------
L2_BYTES = 129e6


def csr_bytes(n, nnz):
    """Algorithmic bytes of one CSR apply: values and column indices once, the
    row pointers, x once, y written once."""
    return 12 * nnz + 4 * (n + 1) + 16 * n


def wilson_bytes(sites, ncols, fp32=False):
    """Algorithmic bytes of one D apply: links (4 x 144 B per site, each read
    once and used by both hops), input and output spinors (192 B each) per
    column; half of that with FP32 data."""
    b = sites * (576 + 384 * ncols)
    return b // 2 if fp32 else b


def workload_name(dims, sources, mixed):
    if tuple(dims) == WL["dims"] and sources == "point" and not mixed:
        return WORKLOAD_NAME
    src = "12 point sources" if sources == "point" else "12 Z4 noise sources (seed 0)"
    prec = ", mixed precision (FP32 iterations, FP64 reliable updates)" if mixed else ""
    return ("wilson-dirac %s kappa=0.155 A=D^H D, %s, seed tol 1e-12 reorth/100, CG tol 1e-8%s"
            % ("x".join(map(str, dims)), src, prec))


def workload_config(dims, sources, mixed, world=1, m_max=None):
    """The `config` object of a solve workload, the same for both arms."""
    return {"workload": workload_name(dims, sources, mixed), "lattice": "x".join(map(str, dims)),
            "n": 12 * int(np.prod(dims)), "nrhs": WL["nrhs"], "precision": "mixed" if mixed else "fp64",
            "kappa": WL["kappa"], "tol_seed": WL["tol_seed"], "reorth_freq": WL["reorth_freq"],
            "reorth_passes": WL["reorth_passes"], "tol_rest": WL["tol_rest"], "m_max": m_max or WL["m_max"],
            "sources": "unit point sources at site 0 (every spin and colour)" if sources == "point"
            else "Z4 noise, seed 0", "links": "exp(0.3 i H), H random Hermitian traceless, seed 0",
            "parallelism": "replicas" if world > 1 else "single-gpu",
            "l2": "flushed (512 MB write) before every step, outside the timed events"}


def run_sweep(args):
    import torch
    from paper_0810_0330_gb300 import binding as S
    from paper_0810_0330_gb300 import inputs as I
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    hbm = MEASURED_PEAKS.get("hbm_gbs", 6663.9)
    pts = []
    for side in (64, 512, 2048, 4096)[:args.sweep_max + 1]:
        rp, ci, v = I.laplacian_2d_csr(side, side)
        n, nnz = side * side, ci.shape[0]
        ctx = S.seed_create_csr(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev),
                                torch.from_numpy(v).to(dev), S.seed_params_default(m_max=4))
        reps = max(20, min(2000, int(2e9 / csr_bytes(n, nnz))))
        ms = S.seed_time_operator(ctx, 0, 1, reps)
        b = csr_bytes(n, nnz)
        pts.append({"op": "csr_spmv", "kernel": "k_csr_spmv", "n": n, "nnz": nnz, "ncols": 1, "ms": ms,
                    "bytes": b, "gbs": b / (ms * 1e-3) / 1e9, "frac_hbm": b / (ms * 1e-3) / 1e9 / hbm,
                    "l2_resident": b < L2_BYTES, "reps": reps})
        S.seed_destroy(ctx)
        del rp, ci, v
    # FP64 and FP32 on L^4, then FP32 only on the two mixed-precision lattice sizes
    lattices = [((L, L, L, L), True) for L in (8, 16, 24)[:args.sweep_max]]
    if args.sweep_max >= 3:
        lattices += [((16, 16, 16, 32), False), ((32, 32, 32, 64), False)]
    for dims, with_fp64 in lattices:
        sites = int(np.prod(dims))
        U = torch.from_numpy(I.random_su3_links(dims, WL["link_eps"], seed=WL["link_seed"])).to(dev)
        ctx = S.seed_create_wilson(dims, WL["kappa"], U, S.seed_params_default(m_max=4))
        for ncols in ((1, 11) if with_fp64 else ()):
            b = wilson_bytes(sites, ncols)
            reps = max(10, min(500, int(4e9 / b)))
            ms = S.seed_time_operator(ctx, 1, ncols, reps)
            fl = FLOPS_PER_SITE_D * sites * ncols
            pts.append({"op": "wilson_D", "kernel": "k_dslash<+1>", "dims": dims, "n": 12 * sites, "ncols": ncols,
                        "ms": ms, "bytes": b, "gbs": b / (ms * 1e-3) / 1e9, "frac_hbm": b / (ms * 1e-3) / 1e9 / hbm,
                        "tflops": fl / (ms * 1e-3) / 1e12, "frac_fp64": fl / (ms * 1e-3) / 1e9 / FP64_PEAK_GFLOPS,
                        "l2_resident": b < L2_BYTES, "reps": reps})
        S.seed_destroy(ctx)
        # the FP32 copy of the operator (mixed-precision iterations): bound by memory traffic
        ctx = S.seed_create_wilson(dims, WL["kappa"], U, S.seed_params_default(m_max=4, precision=1))
        for ncols in (1, 11):
            b = wilson_bytes(sites, ncols, fp32=True)
            reps = max(10, min(500, int(4e9 / b)))
            ms = S.seed_time_operator(ctx, 4, ncols, reps)
            fl = FLOPS_PER_SITE_D * sites * ncols
            pts.append({"op": "wilson_D_fp32", "kernel": fp32_kernel_name(sites) + "<+1>", "dims": dims, "n": 12 * sites,
                        "ncols": ncols, "ms": ms, "bytes": b, "gbs": b / (ms * 1e-3) / 1e9,
                        "frac_hbm": b / (ms * 1e-3) / 1e9 / hbm, "tflops": fl / (ms * 1e-3) / 1e12,
                        "l2_resident": b < L2_BYTES, "reps": reps})
        S.seed_destroy(ctx)
        del U
        torch.cuda.empty_cache()
    for p in pts:
        for k in ("ms", "gbs", "frac_hbm", "tflops", "frac_fp64"):
            if k in p:
                p[k] = round(p[k], 5)
    print(json.dumps({"sweep": pts, "hbm_peak_gbs": hbm, "fp64_peak_tflops": FP64_PEAK_GFLOPS / 1e3,
                      "timing": "mean of back-to-back launches on the same buffers (CUDA events, library stream)"}),
          flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def make_problem(S, I, torch, dev, dims, sources, mixed, m_max, reliable_delta=0.0):
    """Context, sources eta (host and device), B and X blocks of one solve workload."""
    nrhs = WL["nrhs"]
    n = 12 * int(np.prod(dims))
    U = torch.from_numpy(I.random_su3_links(dims, WL["link_eps"], seed=WL["link_seed"])).to(dev)
    prm = S.seed_params_default(m_max=m_max, reorth_freq=WL["reorth_freq"], reorth_passes=WL["reorth_passes"],
                                tol_seed=WL["tol_seed"], tol_rest=WL["tol_rest"], x0_zero=1,
                                precision=1 if mixed else 0, reliable_delta=reliable_delta)
    ctx = S.seed_create_wilson(dims, WL["kappa"], U, prm)
    eta_h = I.point_sources(dims, nrhs) if sources == "point" else I.z4_noise(n, nrhs, seed=0)
    ETA = torch.from_numpy(np.ascontiguousarray(eta_h.T)).to(dev).t()     # (n, nrhs) column-major
    B = torch.empty((nrhs, n), dtype=torch.complex128, device=dev).t()
    X = torch.empty((nrhs, n), dtype=torch.complex128, device=dev).t()
    return dict(ctx=ctx, U=U, eta_h=eta_h, ETA=ETA, B=B, X=X, n=n, vol=int(np.prod(dims)))


def solve_step(S, p):
    """One step of the workload: B = D^H eta, seed solve of system 1, CG on the others."""
    S.seed_apply(p["ctx"], 2, p["ETA"], p["B"])
    i1 = S.seed_solve_first(p["ctx"], p["B"], p["X"])
    i2 = S.seed_solve_rest(p["ctx"], p["B"], p["X"])
    return i1, i2


def time_steps(S, torch, p, flush, steps, warmup, clk=None):
    """Warm-up, then `steps` steps each between CUDA events on the current stream
    (L2 flushed before each, outside the events).  Returns per-step ms and the
    last step's infos."""
    for _ in range(warmup):
        flush.zero_()
        solve_step(S, p)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    infos = None
    for k in range(steps):
        flush.zero_()
        ev[k][0].record()
        infos = solve_step(S, p)
        ev[k][1].record()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], infos


def dslash_roofline(S, ctx, vol, mixed, dims, ncols_total):
    """The dominant kernel, the Wilson hopping kernel, timed live on the
    library's stream: one launch over all CG columns, and the launch shapes the
    CG graphs issue (one per concurrent column branch)."""
    shapes = cg_branch_cols(ncols_total)
    if not mixed:
        k_ms = S.seed_time_operator(ctx, 1, ncols_total, 200)
        flops = FLOPS_PER_SITE_D * vol * ncols_total
        achieved = flops / (k_ms * 1e-3) / 1e12
        peak = FP64_PEAK_GFLOPS / 1e3
        probe = S.seed_time_fma(S.SEED_F64)["tflops"]
        shape_t = {}
        for c in sorted(set(shapes)):
            m = S.seed_time_operator(ctx, 1, c, 200)
            a = FLOPS_PER_SITE_D * vol * c / (m * 1e-3) / 1e12
            shape_t[str(c)] = {"ms_per_launch": round(m, 5), "achieved": round(a, 4), "frac": round(a / peak, 4)}
        return {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4),
                "traffic": dslash_traffic() if tuple(dims) == WL["dims"] and ncols_total == 11 else None,
                "kernel": "k_dslash<+1> (Wilson D, FP64 complex), %d columns in one launch: the work of one CG "
                          "half-iteration" % ncols_total,
                "ms_per_launch": round(k_ms, 5), "flops_per_launch": flops,
                "flops_per_site": FLOPS_PER_SITE_D,
                "epilogue_flops_per_site": FLOPS_PER_SITE_D_EPILOGUE,
                "frac_with_epilogue": round((FLOPS_PER_SITE_D + FLOPS_PER_SITE_D_EPILOGUE) * vol * ncols_total /
                                            (k_ms * 1e-3) / 1e12 / peak, 4),
                "launch_shapes": {"cg_branches": shapes, "per_shape": shape_t},
                "peak_note": "FP64 pipe from unit counts: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz",
                "fp64_instructions_per_site": FP64_INSTR_PER_SITE_D,
                "instruction_mix_ceiling": round(FLOPS_PER_SITE_D / (2.0 * FP64_INSTR_PER_SITE_D), 4),
                "frac_of_instruction_mix_ceiling": round(achieved / peak / (FLOPS_PER_SITE_D /
                                                                             (2.0 * FP64_INSTR_PER_SITE_D)), 4),
                "peak_measured_probe": round(probe, 4), "frac_of_probe": round(achieved / probe, 4),
                "probe": "seed_time_fma(SEED_F64): FMA chains over the whole GPU, this run",
                "fp64_matrix_probe": {k: round(v, 4) for k, v in S.seed_time_fp64_paths().items()}}
    k_ms = S.seed_time_operator(ctx, 4, ncols_total, 200)
    b = wilson_bytes(vol, ncols_total, fp32=True)
    achieved = b / (k_ms * 1e-3) / 1e9
    peak = MEASURED_PEAKS.get("hbm_gbs", 6663.9)
    shape_t = {}
    for c in sorted(set(shapes)):
        m = S.seed_time_operator(ctx, 4, c, 200)
        a = wilson_bytes(vol, c, fp32=True) / (m * 1e-3) / 1e9
        shape_t[str(c)] = {"ms_per_launch": round(m, 5), "achieved": round(a, 1), "frac": round(a / peak, 4)}
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": dslash_traffic(fp32=True) if tuple(dims) == DSLASH32_TRAFFIC_DIMS and ncols_total == 11
            else None,
            "kernel": "%s<+1> (Wilson D, FP32 complex), %d columns in one launch: the work of one CG "
                      "half-iteration" % (fp32_kernel_name(vol), ncols_total),
            "ms_per_launch": round(k_ms, 5), "bytes_per_launch": b, "l2_resident": b < L2_BYTES,
            "launch_shapes": {"cg_branches": shapes, "per_shape": shape_t},
            "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}


def flush_roofline(S, torch, dev, n, steps, nsys):
    """The seeding products of one block flush in mixed precision, G = V_blk^H R_0
    (steps x nsys, FP32 complex vectors of length n) on the tensor cores
    (k_blk_dots_tc through seed_block_products): algorithmic bytes = every
    column read once, against the measured HBM copy peak."""
    g = torch.Generator(device=dev).manual_seed(0)
    V = torch.randn((steps, n), dtype=torch.complex64, device=dev, generator=g).t()
    R = torch.randn((nsys, n), dtype=torch.complex64, device=dev, generator=g).t()
    _, ms = S.seed_block_products(V, R, reps=50)
    b = (steps + nsys) * n * 8
    peak = MEASURED_PEAKS.get("hbm_gbs", 6663.9)
    del V, R
    return {"bound": "hbm", "kernel": "k_blk_dots_tc (tcgen05 kind::tf32, 3xTF32, TMA-staged)",
            "shape": "%d steps x %d systems, n = %d" % (steps, nsys, n), "ms_per_launch": round(ms, 5),
            "bytes_per_launch": b, "achieved": round(b / (ms * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
            "frac": round(b / (ms * 1e-3) / 1e9 / peak, 4)}


def run_secondary(S, I, torch, dev, flush, steps, warmup):
    """The 16^3 x 32 lattice with 12 Z4 noise sources: mixed precision against
    plain FP64 on the same workload, each system's FP64 true residual."""
    dims = (16, 16, 16, 32)
    out = {"workload": "wilson-dirac 16x16x16x32 kappa=0.155 A=D^H D, 12 Z4 noise sources (seed 0), seed tol "
                       "1e-12 reorth/100, CG tol 1e-8; Lanczos basis up to 1000 vectors",
           "steps": steps, "warmup": warmup}
    for mixed in (True, False):
        p = make_problem(S, I, torch, dev, dims, "z4", mixed, m_max=1000)
        ms, (i1, i2) = time_steps(S, torch, p, flush, steps, warmup)
        st = S.seed_get_stats(p["ctx"])
        o = {"ms": round(statistics.mean(ms), 3), "step_ms": [round(x, 3) for x in ms],
             "seed_steps": i1[0]["iters"], "cg_iters": [i["iters"] for i in i2[1:]],
             "true_relres_fp64": [i1[0]["true_relres"]] + [i["true_relres"] for i in i2[1:]],
             "converged": bool(i1[0]["converged"]) and all(i["converged"] for i in i2[1:]),
             "phase_ms": {"seed_solve_first": round(st["ms_seed"], 3), "seed_solve_rest": round(st["ms_rest"], 3)}}
        if mixed:
            o["roofline"] = dslash_roofline(S, p["ctx"], p["vol"], True, dims, WL["nrhs"] - 1)
            o["flush_roofline"] = flush_roofline(S, torch, dev, p["n"], steps=25, nsys=WL["nrhs"] - 1)
        out["mixed" if mixed else "fp64"] = o
        S.seed_destroy(p["ctx"])
        del p
        torch.cuda.empty_cache()
    out["speedup_mixed_over_fp64"] = round(out["fp64"]["ms"] / out["mixed"]["ms"], 3)
    return out


LAP = dict(side=64, nrhs=4, m_max=4096, reorth_freq=1, tol_seed=1e-12, tol_rest=1e-8)


def run_laplacian_line(S, I, torch, dev, flush, steps, warmup, with_oracle=True):
    """The 64x64 Dirichlet Laplacian (n = 4096, real FP64 CSR), 4 Gaussian right-hand
    sides from seed 0: seed solve of system 1 to 1e-12 with full reorthogonalization,
    CG on the other three to 1e-8; GPU time per all-RHS solve (CUDA events), and the
    oracle on the same solve (one thread and all host cores)."""
    rp, ci, v = I.laplacian_2d_csr(LAP["side"], LAP["side"])
    n = LAP["side"] ** 2
    Bh = I.gaussian_rhs(n, LAP["nrhs"], seed=0)
    prm = S.seed_params_default(m_max=LAP["m_max"], reorth_freq=LAP["reorth_freq"], tol_seed=LAP["tol_seed"],
                                tol_rest=LAP["tol_rest"])
    ctx = S.seed_create_csr(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), torch.from_numpy(v).to(dev),
                            prm)
    B = torch.from_numpy(np.ascontiguousarray(Bh.T)).to(dev).t()
    X = torch.empty((LAP["nrhs"], n), dtype=torch.float64, device=dev).t()
    ms = []
    for k in range(warmup + steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        i1 = S.seed_solve_first(ctx, B, X)
        i2 = S.seed_solve_rest(ctx, B, X)
        e1.record()
        torch.cuda.synchronize()
        if k >= warmup:
            ms.append(e0.elapsed_time(e1))
    st = S.seed_get_stats(ctx)
    S.seed_destroy(ctx)
    out = {"workload": "2-d 5-point Dirichlet Laplacian 64x64 (n = 4096, CSR FP64), 4 Gaussian RHS (seed 0); seed "
                       "tol 1e-12 with reorthogonalization every step, CG tol 1e-8",
           "ms": round(statistics.mean(ms), 3), "step_ms": [round(x, 3) for x in ms], "seed_steps": i1[0]["iters"],
           "cg_iters": [i["iters"] for i in i2[1:]],
           "ms_seed": round(st["ms_seed"], 3), "ms_rest": round(st["ms_rest"], 3),
           "converged": bool(i1[0]["converged"]) and all(i["converged"] for i in i2[1:])}
    if with_oracle:
        import oracle
        op = oracle.Operator.csr(rp, ci, v)
        for threads, key in ((1, "oracle_ms_1_thread"), (os.cpu_count() or 1, "oracle_ms_all_cores")):
            used = oracle.set_threads(threads)
            t0 = time.perf_counter()
            oracle.seed_solve_all(op, Bh, m_max=LAP["m_max"], reorth_freq=LAP["reorth_freq"], tol_seed=LAP["tol_seed"],
                                  tol_rest=LAP["tol_rest"])
            out[key] = round((time.perf_counter() - t0) * 1e3, 1)
            out[key.replace("ms", "threads")] = used
        oracle.set_threads(1)
    return out


def matvec_hbm(S, I, torch, dev):
    """The metric's second half, operator-apply bandwidth against the HBM peak,
    where the apply is bound by memory: the CSR SpMV of the 2-d Laplacian
    beyond L2 (2048^2 rows) and the FP32 Wilson D of the mixed path on
    16^3 x 32 (11 columns, the CG launch).  CUDA events, library stream."""
    peak = MEASURED_PEAKS.get("hbm_gbs", 6663.9)
    out = {"peak": peak, "unit": "GB/s", "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    rp, ci, v = I.laplacian_2d_csr(2048, 2048)
    ctx = S.seed_create_csr(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), torch.from_numpy(v).to(dev),
                            S.seed_params_default(m_max=4))
    ms = S.seed_time_operator(ctx, 0, 1, 200)
    b = csr_bytes(2048 * 2048, int(ci.shape[0]))
    out["csr_spmv_laplacian_2048sq"] = {"kernel": "k_csr_spmv (FP64)", "ms_per_launch": round(ms, 5), "bytes": b,
                                        "achieved": round(b / (ms * 1e-3) / 1e9, 1),
                                        "frac": round(b / (ms * 1e-3) / 1e9 / peak, 4)}
    S.seed_destroy(ctx)
    del rp, ci, v
    dims = (16, 16, 16, 32)
    U = torch.from_numpy(I.random_su3_links(dims, WL["link_eps"], seed=WL["link_seed"])).to(dev)
    ctx = S.seed_create_wilson(dims, WL["kappa"], U, S.seed_params_default(m_max=4, precision=1))
    ms = S.seed_time_operator(ctx, 4, WL["nrhs"] - 1, 200)
    b = wilson_bytes(int(np.prod(dims)), WL["nrhs"] - 1, fp32=True)
    out["wilson_d_fp32_16x16x16x32_11cols"] = {"kernel": "k_dslash32_site (FP32)", "ms_per_launch": round(ms, 5),
                                               "bytes": b, "achieved": round(b / (ms * 1e-3) / 1e9, 1),
                                               "frac": round(b / (ms * 1e-3) / 1e9 / peak, 4)}
    S.seed_destroy(ctx)
    del U
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch

    rank, world, local = env_rank()
    dist = None
    if world > 1:
        torch.cuda.set_device(local)
        dist = init_replicas("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_0810_0330_gb300 import binding as S
    from paper_0810_0330_gb300 import inputs as I

    if args.kernel_only and args.csr_side:
        rp, ci, v = I.laplacian_2d_csr(args.csr_side, args.csr_side)
        ctx = S.seed_create_csr(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev),
                                torch.from_numpy(v).to(dev), S.seed_params_default(m_max=4))
        ms = S.seed_time_operator(ctx, 0, 1, args.reps)
        b = csr_bytes(args.csr_side ** 2, ci.shape[0])
        print(json.dumps({"kernel": "k_csr_spmv", "n": args.csr_side ** 2, "nnz": int(ci.shape[0]), "ms": ms,
                          "bytes": b, "gbs": b / (ms * 1e-3) / 1e9}), flush=True)
        S.seed_destroy(ctx)
        return 0
    if args.laplacian_once:
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        r = run_laplacian_line(S, I, torch, dev, flush, 1, 0, with_oracle=False)
        print(json.dumps({"laplacian_once": r["workload"], "ms": r["ms"], "ms_seed": r["ms_seed"],
                          "ms_rest": r["ms_rest"], "seed_steps": r["seed_steps"], "cg_iters": r["cg_iters"]}),
              flush=True)
        return 0
    dims, kappa, nrhs = WL["dims"], WL["kappa"], WL["nrhs"]
    if args.kernel_only and args.dims:
        dims = tuple(int(x) for x in args.dims.split(","))
    if args.lattice:
        dims = tuple(int(x) for x in args.lattice.split(","))
    mixed = args.precision == "mixed"
    default_wl = dims == WL["dims"] and args.sources == "point" and not mixed
    vol = int(np.prod(dims))
    n = 12 * vol
    if args.kernel_only:
        U = torch.from_numpy(I.random_su3_links(dims, WL["link_eps"], seed=WL["link_seed"])).to(dev)
        prm = S.seed_params_default(m_max=4, precision=1 if mixed else 0)
        ctx = S.seed_create_wilson(dims, kappa, U, prm)
        ncols = args.ncols or nrhs - 1
        ms = S.seed_time_operator(ctx, 4 if mixed else 1, ncols, args.reps)
        flops = FLOPS_PER_SITE_D * vol * ncols
        b = wilson_bytes(vol, ncols, fp32=mixed)
        print(json.dumps({"kernel": fp32_kernel_name(vol) if mixed else "k_dslash", "dims": dims, "ncols": ncols, "ms": ms,
                          "tflops": flops / (ms * 1e-3) / 1e12, "gbs": b / (ms * 1e-3) / 1e9}), flush=True)
        S.seed_destroy(ctx)
        return 0
    m_max = WL["m_max"] if dims == WL["dims"] else 1000
    p = make_problem(S, I, torch, dev, dims, args.sources, mixed, m_max, args.reliable_delta)
    ctx = p["ctx"]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2

    if args.once:
        i1, i2 = solve_step(S, p)
        torch.cuda.synchronize()
        st = S.seed_get_stats(ctx)
        print(json.dumps({"once": workload_name(dims, args.sources, mixed), "seed_steps": i1[0]["iters"],
                          "ms_seed": round(st["ms_seed"], 3), "ms_rest": round(st["ms_rest"], 3)}), flush=True)
        S.seed_destroy(ctx)
        return 0
    for _ in range(args.warmup):
        flush.zero_()
        i1, i2 = solve_step(S, p)
    torch.cuda.synchronize()
    assert all(i["converged"] for i in i1[:1] + i2[1:]), (i1[0], i2[1:])

    uuid = None
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        uuid = None
    st0 = S.seed_get_stats(ctx)
    if dist:
        replicas_barrier(dist, "before the timed steps")
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    with ClockSampler(uuid) as clk:
        step_ms, (i1, i2) = time_steps(S, torch, p, flush, args.steps, 0)
    if dist:
        replicas_barrier(dist, "after the timed steps")
    t_wall1 = time.perf_counter()
    st1 = S.seed_get_stats(ctx)
    ms = statistics.mean(step_ms)
    ms = max_over_ranks(ms, dist, dev)
    ok = all(i["converged"] for i in i1[:1] + i2[1:])
    launches = st1["kernel_launches"] - st0["kernel_launches"]

    roof = dslash_roofline(S, ctx, vol, mixed, dims, nrhs - 1)

    # end to end through the public API, host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        eta_pin = torch.from_numpy(np.ascontiguousarray(p["eta_h"].T)).pin_memory()
        x_pin = torch.empty((nrhs, n), dtype=torch.complex128).pin_memory()
        ETA2 = torch.empty((nrhs, n), dtype=torch.complex128, device=dev)
        e2e_ms = []
        for k in range(max(2, args.steps)):
            flush.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ETA2.copy_(eta_pin, non_blocking=True)
            S.seed_apply(ctx, 2, ETA2.t(), p["B"])
            S.seed_solve_first(ctx, p["B"], p["X"])
            S.seed_solve_rest(ctx, p["B"], p["X"])
            x_pin.copy_(p["X"].t(), non_blocking=True)
            b.record()
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
        e2e_v = statistics.mean(e2e_ms)
        e2e_v = max_over_ranks(e2e_v, dist, dev)
        e2e = {"value": round(e2e_v, 3), "unit": "ms", "h2d_bytes_per_step": int(eta_pin.numel() * 16),
               "d2h_bytes_per_step": int(x_pin.numel() * 16), "step_ms": [round(x, 3) for x in e2e_ms]}
    S.seed_destroy(ctx)

    secondary = lap = mv = bat = adj = None
    if rank == 0 and world == 1 and default_wl and not args.no_secondary:
        secondary = run_secondary(S, I, torch, dev, flush, steps=min(args.steps, 3), warmup=1)
        lap = run_laplacian_line(S, I, torch, dev, flush, steps=min(args.steps, 5), warmup=1,
                                 with_oracle=not args.no_cpu_baseline)
        mv = matvec_hbm(S, I, torch, dev)
        del flush
        torch.cuda.empty_cache()
        bat = batched_core(steps=2, warmup=1)
        torch.cuda.empty_cache()
        adj = adjoint_core((16, 16, 16, 16), False, steps=2, warmup=1)
        adj_mixed = adjoint_core((16, 16, 16, 16), True, steps=2, warmup=1)
        adj["mixed_precision_ms"] = adj_mixed["ms"]
        adj["mixed_precision_grad_kappa"] = adj_mixed["grad_kappa"]
        adj["speedup_mixed_over_fp64"] = round(adj["ms"] / adj_mixed["ms"], 3)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and default_wl:
        cpu = cpu_baseline_obj()

    if rank == 0:
        cfg = workload_config(dims, args.sources, mixed, world, m_max)
        if mixed:
            cfg["reliable_delta"] = args.reliable_delta or 0.001
        if secondary is not None:
            cfg["secondary"] = secondary
        if lap is not None:
            cfg["laplacian_64"] = lap
        if bat is not None:
            cfg["batched"] = bat
        if adj is not None:
            cfg["adjoint"] = adj
        out = {"metric": METRIC, "value": round(ms, 3), "unit": "ms", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False,
               "scaling": "weak", "vs_baseline": None,
               "vs_baseline_note": "the paper prints no time for this metric and workload (its timings are "
                                   "CPU-cluster seconds for a 20^3x32 lattice); the oracle's time is in "
                                   "cpu_baseline",
               "dtype": "f32+f64" if mixed else "f64", "data": "synthetic", "config": cfg,
               "run": {"seed_steps": i1[0]["iters"], "cg_iters": [i["iters"] for i in i2[1:]],
                       "true_relres": [i1[0]["true_relres"]] + [i["true_relres"] for i in i2[1:]],
                       "last_step_phase_ms": {"seed_solve_first": round(st1["ms_seed"], 3),
                                              "seed_solve_rest": round(st1["ms_rest"], 3)},
                       "wall_s_timed_region": round(t_wall1 - t_wall0, 3),
                       "step_ms": [round(x, 3) for x in step_ms], "converged": ok},
               "roofline": roof, "matvec_hbm": mv, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
               "clocks": clk.summary()}
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def adjoint_core(dims, mixed, steps, warmup, reorth_freq=None):
    """Loss sum_j ||x_j - t_j||^2, x = A(kappa)^{-1} b through the autograd
    Function: forward (context, seed solve, CG) and backward (adjoint solves
    from zero, the default, and seeded from the forward basis for comparison,
    and the kappa gradient), each timed with CUDA events.  Returns a dict."""
    import torch
    from paper_0810_0330_gb300 import inputs as I
    from paper_0810_0330_gb300.adjoint import WilsonSeedSolve
    dev = torch.device("cuda", torch.cuda.current_device())
    kappa, nrhs = 0.150, 8
    n = 12 * int(np.prod(dims))
    U = torch.from_numpy(I.random_su3_links(dims, WL["link_eps"], seed=WL["link_seed"])).to(dev)
    B = torch.from_numpy(np.ascontiguousarray(I.gaussian_rhs(n, nrhs, seed=0, complex_=True).T)).to(dev).t()
    T = torch.from_numpy(np.ascontiguousarray(I.gaussian_rhs(n, nrhs, seed=1, complex_=True).T)).to(dev).t()
    freq = reorth_freq if reorth_freq is not None else 100
    prm = dict(m_max=1000, reorth_freq=freq, reorth_passes=2, tol_seed=1e-10, tol_rest=1e-8,
               precision=1 if mixed else 0)
    res = {}
    for seeded in ((False,) if mixed else (True, False)):
        fw, bw, its, fits = [], [], [], []
        for step in range(warmup + steps):
            k = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            torch.cuda.synchronize()
            e[0].record()
            X = WilsonSeedSolve.apply(k, B, U, dims, 0, prm, seeded)
            loss = ((X - T).abs() ** 2).sum()
            e[1].record()
            loss.backward()
            e[2].record()
            torch.cuda.synchronize()
            if step >= warmup:
                fw.append(e[0].elapsed_time(e[1]))
                bw.append(e[1].elapsed_time(e[2]))
                its.append(sum(i["iters"] for i in X.grad_fn.info_backward))
                fits.append([i["iters"] for i in X.grad_fn.info_forward])
            del X, loss
        res[seeded] = dict(fw=statistics.mean(fw), bw=statistics.mean(bw), bw_iters=its[-1], fw_iters=fits[-1],
                           grad_kappa=float(k.grad))
    s_, u_ = res.get(True, res[False]), res[False]
    # the value is the library's default, the backward solves started from zero
    return {"ms": round(u_["fw"] + u_["bw"], 3),
            "workload": "wilson-dirac %s kappa=%.3f A=D^H D, %d Gaussian b and t (seeds 0, 1), seed tol 1e-10 "
                        "reorth/%d, CG tol 1e-8%s" % ("x".join(map(str, dims)), kappa, nrhs, freq,
                                                      ", mixed precision" if mixed else ""),
            "backward": "unseeded (default)", "forward_ms": round(u_["fw"], 3),
            "backward_unseeded_ms": round(u_["bw"], 3), "backward_seeded_ms": round(s_["bw"], 3),
            "backward_cg_iters_seeded": s_["bw_iters"], "backward_cg_iters_unseeded": u_["bw_iters"],
            "forward_iters": s_["fw_iters"], "grad_kappa": u_["grad_kappa"],
            "grad_kappa_seeded": s_["grad_kappa"], "steps": steps, "warmup": warmup}


def run_adjoint(args):
    import torch
    torch.cuda.set_device(0)
    dims = tuple(int(x) for x in args.lattice.split(",")) if args.lattice else (16, 16, 16, 16)
    r = adjoint_core(dims, args.precision == "mixed", args.steps, args.warmup, args.reorth_freq)
    out = {"metric": "adjoint forward+backward time (loss and gradients for b and kappa)", "value": r["ms"],
           "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
           "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic", "config": r}
    print(json.dumps(out), flush=True)
    return 0


def batched_core(steps, warmup):
    """All right-hand sides of 32 independent problems: one after another
    through seed_solve_first / seed_solve_rest, against seed_batch_solve (all
    problems concurrently), FP64 and mixed precision; CUDA events around each
    whole batch on the current stream (the library orders its streams after it)."""
    import torch
    from paper_0810_0330_gb300 import binding as S
    from paper_0810_0330_gb300 import inputs as I
    dev = torch.device("cuda", torch.cuda.current_device())
    probs = I.batch_problems(count=32, n_min=1e4, n_max=1e6, seed=0)
    prm = dict(m_max=500, reorth_freq=100, reorth_passes=2, tol_seed=1e-10, tol_rest=1e-8)
    arrays = []
    for p in probs:
        rp, ci, v, B = I.batch_problem_arrays(p)
        arrays.append((torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), torch.from_numpy(v).to(dev),
                       torch.from_numpy(np.ascontiguousarray(B.T)).to(dev).t()))
    Xs = [torch.zeros_like(a[3].t()).t() for a in arrays]

    def contexts(**kw):
        return [S.seed_create_csr(a[0], a[1], a[2], S.seed_params_default(**prm, **kw)) for a in arrays]

    def timed(fn):
        ms = []
        for step in range(warmup + steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            if step >= warmup:
                ms.append(e0.elapsed_time(e1))
        return statistics.mean(ms), out

    ctx64 = contexts()

    def sequential():
        its = []
        for c, a, X in zip(ctx64, arrays, Xs):
            i1 = S.seed_solve_first(c, a[3], X)
            i2 = S.seed_solve_rest(c, a[3], X)
            its.append((i1[0]["iters"], sum(i["iters"] for i in i2[1:]), all(i["converged"] for i in i2[1:])))
        return its

    seq_ms, seq_its = timed(sequential)
    bat_ms, bat_info = timed(lambda: S.seed_batch_solve(ctx64, [a[3] for a in arrays], Xs))
    for c in ctx64:
        S.seed_destroy(c)
    ctx32 = contexts(precision=1)
    mix_ms, mix_info = timed(lambda: S.seed_batch_solve(ctx32, [a[3] for a in arrays], Xs))
    for c in ctx32:
        S.seed_destroy(c)
    ok = all(all(i["converged"] for i in inf[1:]) for inf in bat_info + mix_info)
    return {"ms": round(bat_ms, 3),
            "workload": "32 shifted 2-d/3-d Dirichlet Laplacians (shift U(0.01,1)), n log-uniform 1e4..1e6, 4..16 "
                        "Gaussian RHS each (seed 0); seed tol 1e-10 reorth/100, CG tol 1e-8",
            "total_n": int(sum(a[0].shape[0] - 1 for a in arrays)), "total_rhs": int(sum(p["nrhs"] for p in probs)),
            "sequential_ms": round(seq_ms, 3), "batched_fp64_ms": round(bat_ms, 3),
            "batched_mixed_ms": round(mix_ms, 3), "speedup_batched_fp64": round(seq_ms / bat_ms, 3),
            "speedup_batched_mixed": round(seq_ms / mix_ms, 3), "converged": ok,
            "seed_steps": [i[0] for i in seq_its], "steps": steps, "warmup": warmup}


def run_batched(args):
    import torch
    torch.cuda.set_device(0)
    r = batched_core(args.steps, args.warmup)
    out = {"metric": "batched uneven problems: all right-hand sides of 32 problems", "value": r["ms"],
           "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
           "dtype": "f64", "data": "synthetic", "config": r}
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.sweep:
        return run_sweep(args)
    if args.batched:
        return run_batched(args)
    if args.adjoint:
        return run_adjoint(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
