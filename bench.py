#!/usr/bin/env python3
"""Benchmark of the PNOF7 energy + orbital-Lagrangian build on GB300.

One step = one build (E, lambda, dE/dgamma) plus its adjoint (dE/dC) of the large
workload: nbf 1200, naux 4800, 50 pairs, Ncwo 2 (150 active orbitals), packed B,
mixed precision, inputs resident in HBM (the 27.6 GB split copy of B that each build
streams is far larger than L2).  Prints one JSON line.  Under torchrun (--gpus N) the
ranks share each build: the auxiliary index is sharded over them and one NCCL all-reduce
of the partial sums J, K and the two-electron G finishes it (strong scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Lagrangian builds/sec & TFLOP/s, mixed vs FP64 GPU path at ≤1e-6 Eh"
UNIT = "builds/s"
WORKLOADS = {
    "large": dict(nbf=1200, naux=4800, npair=50, ncwo=2, packed=True),
    "precision": dict(nbf=500, naux=2000, npair=20, ncwo=3, packed=False),
}
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=list(WORKLOADS))
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-loop", action="store_true",
                    help="skip the timing of the optimisation procedure (Sec. III.D)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--naux", type=int, default=0,
                    help="override naux (profiling captures on a slice of the workload)")
    return ap.parse_args()


def flops_build(N, Q, A):
    """Algorithmic flops of one build: X = B C (2QN^2A), b = C^T X (2QNA^2),
    G += X Y (2QNA^2), h C and lambda = C^T G (2N^2A each)."""
    return 2.0 * Q * N * A * (N + 2 * A) + 4.0 * N * N * A


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, ws, device):
    """The slowest rank's time (the whole job's clock): all-reduce MAX over the process
    group when there is more than one rank."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as tdist
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return t.item()


def job_rate(ms_max, builds_per_step=1):
    """Whole-job builds/s over the slowest rank's step time.  Under torchrun the ranks share
    one build per step (its auxiliary index sharded over them), so builds_per_step is 1."""
    return builds_per_step * 1e3 / ms_max


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
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
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- inputs
def make_inputs(w, seed, dev, P0=0, P1=None):
    """The workload's inputs on the device; of B only the auxiliary slices [P0, P1)."""
    import numpy as np
    import torch

    import synth
    N, Q = w["nbf"], w["naux"]
    P1 = Q if P1 is None else P1
    prob = synth.Problem(N, Q, w["npair"], w["ncwo"], seed)
    d = synth.generate(prob, with_B=False)
    npk = N * (N + 1) // 2
    nloc = P1 - P0
    B = torch.empty((nloc, npk) if w["packed"] else (nloc, N, N), dtype=torch.float64,
                    device=dev)
    chunk = 160
    for p0 in range(P0, P1, chunk):
        p1 = min(P1, p0 + chunk)
        host = synth.gen_B(seed, Q, N, packed=w["packed"], p0=p0, p1=p1)
        B[p0 - P0:p1 - P0].copy_(torch.from_numpy(host))
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    return prob, d, dict(B=B, h=t(d["h"]), C=t(d["C"]), gamma=t(d["gamma"]),
                         pair_map=t(d["pair_map"].astype(np.int32)))


# ----------------------------------------------------------------------------- CPU oracle
def oracle_streamed_build(w, seed, nsteps=1, on_step=None):
    """One full FP64 oracle build of the workload (E, lambda, dE/dgamma, dE/dC), its operator
    route streamed over nsteps blocks of auxiliary slices (oracle.pnof.build_streamed).  The
    inputs are regenerated block by block outside the timed parts.  Returns (result, list
    of per-block oracle seconds; the last one includes the work after the final block)."""
    import numpy as np

    import synth
    from oracle import pnof
    N, Q = w["nbf"], w["naux"]
    prob = synth.Problem(N, Q, w["npair"], w["ncwo"], seed)
    d = synth.generate(prob, with_B=False)
    bounds = [Q * k // nsteps for k in range(nsteps + 1)]
    ready, done = [], []

    def blocks():
        for k in range(nsteps):
            blk = synth.gen_B(seed, Q, N, packed=False, p0=bounds[k], p1=bounds[k + 1])
            ready.append(time.perf_counter())
            yield blk

    def mark(_n):
        done.append(time.perf_counter())
        if on_step is not None:
            on_step(len(done), done[-1] - ready[-1])

    res = pnof.build_streamed(d["h"], blocks(), d["C"], d["gamma"], d["pair_map"], prob.npair,
                              prob.ncwo, pnof.PNOF7, on_block=mark)
    t_end = time.perf_counter()
    steps = [b - a for a, b in zip(ready, done)]
    steps[-1] += t_end - done[-1]
    return res, np.array(steps)


def oracle_block_sample(w, seed, k, nblk):
    """Untimed warm-up work for the reference arm: the oracle's AO operators on block k of
    nblk blocks of auxiliary slices."""
    import synth
    from oracle import pnof
    N, Q = w["nbf"], w["naux"]
    prob = synth.Problem(N, Q, w["npair"], w["ncwo"], seed)
    d = synth.generate(prob, with_B=False)
    p0, p1 = Q * k // nblk, Q * (k + 1) // nblk
    blk = synth.gen_B(seed, Q, N, packed=False, p0=p0, p1=p1)
    pnof.ao_operators(blk, d["C"][:, :prob.nact])


def oracle_small_medians(reps=5):
    """Builds/s of the FP64 oracle on the plain, differentiation and precision workloads:
    the median of `reps` timed builds each (inputs generated beforehand)."""
    import numpy as np

    import synth
    from oracle import pnof
    out = {}
    for name in ("plain", "differentiation", "precision"):
        prob, packed = synth.config_problem(name)
        d = synth.generate(prob, packed=packed)
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            pnof.build(d["h"], d["B"], d["C"], d["gamma"], d["pair_map"], prob.npair, prob.ncwo,
                       pnof.PNOF7, packed=packed)
            ts.append(time.perf_counter() - t0)
        med = float(np.median(ts))
        out[name] = {"shape": f"{prob.nbf}/{prob.naux}/{prob.npair}/{prob.ncwo}",
                     "builds_per_s": 1.0 / med, "median_s": med, "runs": reps}
    return out


def blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(i.get("num_threads", 1) for i in info)
    except Exception:
        pass
    return os.cpu_count()


def split_b_bytes(Q, N):
    """Bytes of the split B the half transform streams: per slice the stored lower triangle
    of 128-row tiles (the last tile's rows rounded up to 64), two fp16 planes."""
    T = (N + 127) // 128
    R_last = (N - 128 * (T - 1) + 63) // 64 * 64
    per_slice = 16384 * (T - 1) * T // 2 + R_last * (128 * (T - 1) + R_last)
    return Q * per_slice * 4


def tensor_peak(pk, region_s, clk):
    """(kind, dense fp16 TFLOP/s) for the roofline: the burst peak for a timed region
    shorter than 2 s whose SM clock median stays within 5 % of its maximum (the kernel then
    runs at full clocks, as the burst GEMM did), the sustained peak (seconds of back-to-back
    GEMMs under the power cap) otherwise."""
    mhz, mhz_max = (clk or {}).get("sm_mhz"), (clk or {}).get("sm_max_mhz")
    capped = bool(mhz and mhz_max and mhz < 0.95 * mhz_max)
    kind = "sustained" if (region_s >= 2.0 or capped) else "burst"
    key = "bf16_tflops_sustained" if kind == "sustained" else "bf16_tflops"
    return kind, pk.get(key, FALLBACK_PEAKS[key])


# ----------------------------------------------------------------------------- traffic record
def recorded_traffic(kernel_src):
    """Per-launch DRAM bytes of the half-transform kernel from the committed ncu summary,
    or None when the summary is missing or the kernel source changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "half_transform_large.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_sha = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", txt)
    m_b = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m_sha or not m_b:
        return None
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
    return float(m_b.group(1)) if sha == m_sha.group(1) else None


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 CPU oracle on the host cores, the same workload as our arm.  The K timed steps
    together are exactly one full build: step k runs the oracle's operator route on block k of
    K blocks of auxiliary slices (the last step also the work after the final block), so
    value = 1 build / (sum of the step times), with nothing extrapolated.  Warm-up: W blocks,
    untimed.  Rank 0 only under torchrun."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    for k in range(args.warmup):
        oracle_block_sample(w, args.seed, k % args.steps, args.steps)
    _, steps = oracle_streamed_build(w, args.seed, nsteps=args.steps)
    total = float(steps.sum())
    value = 1.0 / total
    cores = blas_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: nbf={w['nbf']}, naux={w['naux']}, "
                               f"npair={w['npair']}, ncwo={w['ncwo']}, PNOF7, FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"one full build of the workload, its {w['naux']} auxiliary "
                                   f"slices streamed in {args.steps} blocks, one block per "
                                   "step (the last step also forms J, K, E, G, lambda and "
                                   "dE/dgamma); input generation untimed",
                         "step_s": [round(float(x), 3) for x in steps]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as tdist

    ws, rank, local = dist_env()
    if ws > 1:
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2004_06142_gb300 import build as libbuild
    libbuild.build()
    import paper_2004_06142_gb300 as dn

    w = dict(WORKLOADS[args.workload])
    if args.naux:
        w["naux"] = args.naux
    N, Q = w["nbf"], w["naux"]
    # with several ranks the auxiliary index is sharded: rank r holds slices [P0, P1) of B,
    # builds its partial sums, and one all-reduce (NCCL) of J, K and the two-electron G
    # precedes the finish on every rank (Sec. III.D: these are sums over P)
    P0, P1 = dn.shard_range(Q, rank, ws)
    Qloc = P1 - P0
    prob, host, x = make_inputs(w, args.seed, dev, P0, P1)
    A = prob.nact
    layout = dn.B_PACKED if w["packed"] else dn.B_DENSE

    def barrier():
        if ws > 1:
            tdist.barrier()

    mixed = dn.Builder(N, Qloc, prob.npair, prob.ncwo, dn.PNOF7, layout, dn.MIXED, device=dev)
    mixed.prepare(x["B"])
    mixed.autotune(x["h"], x["C"], x["gamma"], x["pair_map"])
    Ebar = torch.ones(1, dtype=torch.float64, device=dev)

    def forward(C, g):
        if ws > 1:
            return mixed.forward_sharded(x["h"], C, g, x["pair_map"])
        return mixed.forward(x["h"], C, g, x["pair_map"])

    def step():
        E, lam, dEdg = forward(x["C"], x["gamma"])
        dC, dg = mixed.backward(Ebar)
        return E, lam, dEdg, dC

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert mixed.status() == 0, "device status after warm-up"

    # ---------------- timed region (device resident inputs)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    dn.donof_profile_enable(True)
    launches0 = dn.donof_launch_count()
    # one event per step boundary on the launching stream (the library launches on torch's
    # current stream): the total over K steps gives `value`, the per-step times the median
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record()
    for k in range(args.steps):
        out = step()
        evs[k + 1].record()
    torch.cuda.synchronize()
    barrier()
    launches = dn.donof_launch_count() - launches0
    clk = clocks.stop()
    ms = evs[0].elapsed_time(evs[-1]) / args.steps
    step_ms = sorted(evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps))
    ms_median = step_ms[len(step_ms) // 2] if args.steps % 2 else \
        0.5 * (step_ms[args.steps // 2 - 1] + step_ms[args.steps // 2])
    phases = {}
    for i, nm in enumerate(dn.PHASES):
        t, n = dn.donof_profile_read(i)
        if n:
            phases[nm] = {"ms_per_launch": t / n, "intervals": n}
    dn.donof_profile_enable(False)
    ms_max = max_over_ranks(ms, ws, dev)
    value = job_rate(ms_max)
    E_mixed = out[0].item()
    res_mixed = [t.detach().cpu().numpy() for t in out]

    # ---------------- end to end through the public API with pinned host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hC, hg = pin(host["C"]), pin(host["gamma"])
    oE = torch.empty(1, dtype=torch.float64).pin_memory()
    olam = torch.empty(N, N, dtype=torch.float64).pin_memory()
    odg = torch.empty(prob.ngamma, dtype=torch.float64).pin_memory()
    odC = torch.empty(N, N, dtype=torch.float64).pin_memory()
    Cd, gd = torch.empty_like(x["C"]), torch.empty_like(x["gamma"])
    h2d = hC.numel() * 8 + hg.numel() * 8
    d2h = (oE.numel() + olam.numel() + odg.numel() + odC.numel()) * 8

    # one GPU: the C-ABI call on host buffers (donof_energy_lagrangian_host: the copies, the
    # build, the adjoint and the copies back in one call); several: the sharded build with
    # the copies around it
    staging = None
    if ws == 1:
        staging = dn.alloc_workspace(dn.donof_host_staging_size(mixed.prob), dev)

    def e2e_step():
        if ws == 1:
            dn.donof_energy_lagrangian_host(mixed.prob, x["h"], mixed.B, hC, hg, x["pair_map"],
                                            mixed.ws, staging, oE, olam, odg, odC)
            return
        Cd.copy_(hC, non_blocking=True)
        gd.copy_(hg, non_blocking=True)
        E, lam, dEdg = forward(Cd, gd)
        dC, _ = mixed.backward(Ebar)
        oE.copy_(E, non_blocking=True)
        olam.copy_(lam, non_blocking=True)
        odg.copy_(dEdg, non_blocking=True)
        odC.copy_(dC, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(args.steps):
        e2e_step()
    f1.record()
    torch.cuda.synchronize()
    barrier()
    ms_e2e = max_over_ranks(f0.elapsed_time(f1) / args.steps, ws, dev)
    assert abs(oE.item() - E_mixed) < 1e-9

    # ---------------- the batched workload: 64 uneven instances in one graph launch
    batch = None
    if not args.no_batch and ws == 1:
        batch = run_batch(dn, dev, args.steps, args.warmup)
        batch["small_workloads"] = run_small_workloads(dn, dev, args.steps, args.warmup)

    # ---------------- the optimisation procedure around the build (occupation optimisation +
    # orbital iterations), mixed builds, on copies of C and gamma
    loop = None
    if not args.no_loop and ws == 1:
        kw = dict(diis_depth=6, zeta=1.0, delta=1e-12, eps_energy=0.0, occ_max_iter=200,
                  occ_gtol=1e-10)
        Cl, gl = x["C"].clone(), x["gamma"].clone()
        mixed.optimize(x["h"], Cl, gl, x["pair_map"], max_outer=1, max_inner=1, **kw)  # warm-up
        Cl, gl = x["C"].clone(), x["gamma"].clone()
        torch.cuda.synchronize()
        dn.donof_profile_enable(True)
        t0 = time.perf_counter()
        res, _ = mixed.optimize(x["h"], Cl, gl, x["pair_map"], max_outer=2, max_inner=4, **kw)
        wall = (time.perf_counter() - t0) * 1e3
        step_ms, nstep = dn.donof_profile_read(dn.PHASES.index("orbital_step"))
        occ_ms, nocc = dn.donof_profile_read(dn.PHASES.index("occ_opt"))
        dn.donof_profile_enable(False)
        loop = {"workload": "2 outer iterations (occupation optimisation, then 4 orbital "
                            "iterations each: zeta 1, DIIS depth 6), symmetrised-lambda start, "
                            "mixed builds, large workload",
                "ms_total": wall, "builds": res["builds"], "orbital_iterations": res["inner"],
                "ms_per_orbital_step": step_ms / max(nstep, 1),
                "ms_per_occupation_optimisation": occ_ms / max(nocc, 1),
                "ms_per_build": ms,
                "E_final": res["E"], "max_asym_final": res["max_asym"],
                "note": "host wall time around the synchronous donof_optimize call (after a "
                        "warm-up call); device time of its parts from the tracing phases: an "
                        "orbital step = F, its AO form, DIIS, the FP64 eigensolver and the "
                        "reorthonormalisation"}
        del Cl, gl

    # ---------------- the plain FP64 GPU path on the same inputs
    fp64 = None
    if not args.no_fp64 and ws == 1:
        del mixed
        torch.cuda.empty_cache()
        b64 = dn.Builder(N, Q, prob.npair, prob.ncwo, dn.PNOF7, layout, dn.FP64,
                         x_budget_bytes=16 << 30, device=dev)
        b64.prepare(x["B"])

        def step64():
            E, lam, dEdg = b64.forward(x["h"], x["C"], x["gamma"], x["pair_map"])
            dC, _ = b64.backward(Ebar)
            return E, lam, dEdg, dC

        step64()
        torch.cuda.synchronize()
        dn.donof_profile_enable(True)
        step64()
        torch.cuda.synchronize()
        half64 = dn.donof_profile_read(dn.PHASES.index("half_transform"))
        dn.donof_profile_enable(False)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        for _ in range(args.fp64_steps):
            o64 = step64()
        g1.record()
        torch.cuda.synchronize()
        ms64 = g0.elapsed_time(g1) / args.fp64_steps
        r64 = [t.detach().cpu().numpy() for t in o64]
        # the hand-off to the orbital update (Eq. Fockian + double eigensolver + rotation)
        Fdiag = -torch.arange(N, dtype=torch.float64, device=dev)
        Cn = torch.empty(N, N, dtype=torch.float64, device=dev)
        epsv = torch.empty(N, dtype=torch.float64, device=dev)
        wsu = dn.donof_orbital_update(o64[1], Fdiag, x["C"], Cn, epsv)
        torch.cuda.synchronize()
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record()
        for _ in range(3):
            dn.donof_orbital_update(o64[1], Fdiag, x["C"], Cn, epsv, ws=wsu)
        u1.record()
        torch.cuda.synchronize()
        upd_ms = u0.elapsed_time(u1) / 3
        # the eigensolver alone on the same F (donof_eigh; eigenvalues and V in place)
        Fm = torch.randn(N, N, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(5))
        Fm = Fm + Fm.T
        Vm = torch.empty_like(Fm)
        wse = dn.donof_eigh(Fm, Vm, epsv)
        torch.cuda.synchronize()
        u0.record()
        for _ in range(3):
            dn.donof_eigh(Fm, Vm, epsv, ws=wse)
        u1.record()
        torch.cuda.synchronize()
        eigh_ms = u0.elapsed_time(u1) / 3
        del Fm, Vm, wse
        # measured FP64 peak: a cuBLAS DGEMM (library routine, for the denominator only)
        Ad = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
        Bd = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
        for _ in range(2):
            torch.matmul(Ad, Bd)
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record()
        for _ in range(5):
            torch.matmul(Ad, Bd)
        d1.record()
        torch.cuda.synchronize()
        dgemm_tf = 5 * 2.0 * 4096 ** 3 / (d0.elapsed_time(d1) * 1e-3) / 1e12
        del Ad, Bd
        half64_ms = half64[0]  # one profiled build: the sum over its P blocks
        half64_tf = 2.0 * Q * N * N * A / (half64_ms * 1e-3) / 1e12
        fp64 = {
            "builds_per_s": 1e3 / ms64, "ms_per_build": ms64,
            "roofline": {"bound": "fp64", "kernel": "k_dgemm (half transform X = B C_act, FP64)",
                         "achieved": half64_tf, "peak": dgemm_tf, "unit": "TFLOP/s",
                         "frac": half64_tf / dgemm_tf, "half_transform_ms": half64_ms,
                         "peak_note": "measured: cuBLAS DGEMM 4096^3 on this GPU"},
            "tflops_algorithmic": flops_build(N, Q, A) / (ms64 * 1e-3) / 1e12,
            "speedup_mixed_over_fp64": ms64 / ms,
            "mixed_minus_fp64": {
                "E_abs": float(abs(res_mixed[0][0] - r64[0][0])),
                "lambda_maxabs": float(np.abs(res_mixed[1] - r64[1]).max()),
                "dE_dgamma_maxabs": float(np.abs(res_mixed[2] - r64[2]).max()),
                "dE_dC_maxabs": float(np.abs(res_mixed[3] - r64[3]).max()),
            },
            "status": b64.status(),
            "orbital_update_ms": upd_ms,
            "eigh_ms": eigh_ms,
        }

    # ---------------- errors against the FP64 oracle's stored values (large workload)
    oracle_err = None
    gpath = os.path.join(ROOT, "tests", "golden", f"large_seed{args.seed}.npz")
    if args.workload == "large" and not args.naux and os.path.exists(gpath):
        z = np.load(gpath)
        oracle_err = {"source": f"tests/golden/large_seed{args.seed}.npz (FP64 oracle, streamed)"}
        paths = [("mixed", res_mixed)] + ([("fp64", r64)] if fp64 else [])
        for nm, r in paths:
            oracle_err[nm] = {
                "E_abs": float(abs(r[0][0] - z["E"][0])),
                "lambda_maxabs": float(np.abs(r[1][:, :A] - z["lam_act"]).max()),
                "dE_dgamma_maxabs": float(np.abs(r[2] - z["dE_dgamma"]).max()),
                "dE_dC_maxabs": float(np.abs(r[3][:, :A] - z["dE_dC_act"]).max()),
            }

    # ---------------- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1:
        _, steps = oracle_streamed_build(w, args.seed, nsteps=20)
        cpu = {"value": 1.0 / float(steps.sum()), "unit": UNIT, "cores": blas_threads(),
               "kind": "oracle",
               "sample": f"one full build of the workload ({float(steps.sum()):.1f} s), the "
                         f"{Q} auxiliary slices streamed in 20 blocks; input generation "
                         "untimed",
               "small_workloads_median_of_5": oracle_small_medians(5)}

    # ---------------- roofline of the dominant kernel (half transform X = B C)
    pk, src = peaks()
    region_s = args.steps * ms * 1e-3
    mhz, mhz_max = (clk or {}).get("sm_mhz"), (clk or {}).get("sm_max_mhz")
    kind, peak_f16 = tensor_peak(pk, region_s, clk)
    half = phases.get("half_transform", {}).get("ms_per_launch")
    roof = None
    if half:
        flops_half = 2.0 * Qloc * N * N * A
        hbm_bytes = split_b_bytes(Qloc, N) + Qloc * N * ((A + 15) // 16 * 16) * 8
        achieved = flops_half / (half * 1e-3) / 1e12
        peak_eff = peak_f16 / 4.0
        traffic = recorded_traffic(os.path.join(ROOT, "paper_2004_06142_gb300", "csrc", "tc.cu"))
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak_eff, "unit": "TFLOP/s",
                "frac": achieved / peak_eff, "traffic": traffic,
                "kernel": "k_tc_gemm<64> (half transform X = B C_act)",
                "peak_note": f"{src} dense fp16 {kind} {peak_f16} TFLOP/s (timed region "
                             f"{region_s:.2f} s, SM clock median {mhz} of {mhz_max} MHz) / 4 "
                             "tensor products per algorithmic product (h*h + h*f + f*h + f*f "
                             "of the integer + fraction split)",
                "issued_tflops": 4 * 2.0 * Qloc * N * N * ((A + 15) // 16 * 16) / (half * 1e-3) / 1e12,
                "frac_of_peak_algorithmic": achieved / peak_f16,
                "hbm_gbs": hbm_bytes / (half * 1e-3) / 1e9,
                "hbm_peak_gbs": pk.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]),
                "hbm_frac": hbm_bytes / (half * 1e-3) / 1e9 / pk.get("hbm_gbs",
                                                                     FALLBACK_PEAKS["hbm_gbs"]),
                "hbm_note": "algorithmic bytes = the stored lower triangle of the split B "
                            "read once (4 B per element, tiles of 128) + the two X outputs "
                            "(8 B per element, nact padded to 16)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "ms_per_step_median": ms_median,
            "timing_note": "value = K steps / their total CUDA-event time (mean step); "
                           "ms_per_step_median = the median of the per-step event times",
            "higher_is_better": True,
            "scaling": "strong" if ws > 1 else "weak", "vs_baseline": None,
            "dtype": "f16 integer+fraction split operands (4 products, exact integer "
                     "accumulation) for X, b and G; fp32 J/K/Y; f64 reductions and outputs",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: nbf={N}, naux={Q}, npair={prob.npair}, "
                                   f"ncwo={prob.ncwo} (nact {A}), "
                                   f"{'packed' if w['packed'] else 'dense'} B, PNOF7, "
                                   "E + lambda + dE/dgamma + dE/dC per step",
                       "l2": "inputs larger than L2 (the split B's stored triangle, "
                             f"{split_b_bytes(Q, N) / 1e9:.1f} GB, "
                             "streamed per build)",
                       "parallelism": (f"auxiliary index sharded over {ws} GPUs ({Qloc} slices "
                                       "on rank 0), one NCCL all-reduce of J, K and the "
                                       "two-electron G per build") if ws > 1 else "single GPU"},
            "tflops_algorithmic": flops_build(N, Q, A) / (ms_max * 1e-3) / 1e12,
            "phases_ms": {k: v["ms_per_launch"] for k, v in phases.items()},
            "fp64_path": fp64,
            "oracle_errors": oracle_err,
            "optimisation_loop": loop,
            "batch_workload": batch,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": job_rate(ms_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "note": "per step: C and gamma host->device, E, lambda, dE/dgamma, dE/dC "
                            "device->host from and to page-locked host buffers; one GPU: one "
                            "C-ABI call (donof_energy_lagrangian_host) per step; B and h stay "
                            "resident (fixed across orbital iterations)"},
            "gpu_launches": launches,
            "clocks": clk,
            "peaks_source": src,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        tdist.destroy_process_group()


def run_small_workloads(dn, dev, steps, warmup):
    """The plain, differentiation and precision workloads (nbf/naux/npair/Ncwo 24/96/5/1,
    120/480/8/4, 500/2000/20/3): one mixed build + adjoint per step, captured once into a
    CUDA graph and replayed (small builds are launch-bound), CUDA events over the replays."""
    import numpy as np
    import torch

    import synth
    out = {}
    for name in ("plain", "differentiation", "precision"):
        c = synth.CONFIGS[name]
        prob = synth.Problem(c["nbf"], c["naux"], c["npair"], c["ncwo"], 0)
        d = synth.generate(prob)
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
        h, B, C, g = t(d["h"]), t(d["B"]), t(d["C"]), t(d["gamma"])
        pm = t(d["pair_map"].astype(np.int32))
        b = dn.Builder(prob.nbf, prob.naux, prob.npair, prob.ncwo, dn.PNOF7, dn.B_DENSE,
                       dn.MIXED, device=dev)
        b.prepare(B)
        Ebar = torch.ones(1, dtype=torch.float64, device=dev)
        st = torch.cuda.Stream(device=dev)
        st.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(st):
            for _ in range(max(3, warmup)):
                b.forward(h, C, g, pm)
                b.backward(Ebar)
        torch.cuda.current_stream(dev).wait_stream(st)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            b.forward(h, C, g, pm)
            b.backward(Ebar)
        graph.replay()
        torch.cuda.synchronize()
        reps = max(20, 10 * steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        assert b.status() == 0
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"shape": f"{prob.nbf}/{prob.naux}/{prob.npair}/{prob.ncwo}",
                     "builds_per_s": 1e3 / ms, "ms_per_build": ms,
                     "tflops_algorithmic": flops_build(prob.nbf, prob.naux, prob.nact)
                     / (ms * 1e-3) / 1e12, "graph_replay": True}
        del b, graph
        torch.cuda.empty_cache()
    return out


def run_batch(dn, dev, steps, warmup, ninst=64):
    """Dissociation-scan-shaped batch: instance i has seed i, nbf ~ U{40..240}, naux = 4 nbf,
    5 pairs, Ncwo ~ U{1..4}; PNOF7, mixed precision, forward + adjoint, one CUDA-graph replay
    per step."""
    import numpy as np
    import torch

    import synth
    probs = synth.batch_problems(ninst)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    cprobs, tens = [], []
    flops = 0.0
    for pr in probs:
        d = synth.generate(pr)
        cprobs.append(dn.make_problem(pr.nbf, pr.naux, pr.npair, pr.ncwo, dn.PNOF7, dn.B_DENSE,
                                      dn.MIXED))
        f64 = torch.float64
        tens.append(dict(h=t(d["h"]), B=t(d["B"]), C=t(d["C"]), gamma=t(d["gamma"]),
                         pair_map=t(d["pair_map"].astype(np.int32)),
                         E=torch.empty(1, dtype=f64, device=dev),
                         lam=torch.empty(pr.nbf, pr.nbf, dtype=f64, device=dev),
                         dE_dgamma=torch.empty(pr.ngamma, dtype=f64, device=dev),
                         dE_dC=torch.empty(pr.nbf, pr.nbf, dtype=f64, device=dev)))
        flops += flops_build(pr.nbf, pr.naux, pr.nact)
    b = dn.Batch(cprobs, tens, device=dev)
    b.prepare()
    flags = dn.BATCH_BACKWARD | dn.BATCH_GRAPH
    for _ in range(max(1, warmup)):
        b.run(flags)
    torch.cuda.synchronize()
    l0 = dn.donof_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        b.run(flags)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    nb = [pr.nbf for pr in probs]
    return {"workload": f"{ninst} instances, nbf {min(nb)}..{max(nb)} (seeds 0..{ninst - 1}), "
                        "naux = 4 nbf, 5 pairs, Ncwo 1..4, PNOF7, mixed, forward + adjoint",
            "builds_per_s": ninst * 1e3 / ms, "ms_per_batch": ms,
            "tflops_algorithmic": flops / (ms * 1e-3) / 1e12,
            "graph_launches_per_step": 1,
            "kernels_per_step": (dn.donof_launch_count() - l0) // steps}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
