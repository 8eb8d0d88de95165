#!/usr/bin/env python
"""Benchmark of the exact-diagonalization hot path on GB300.

Workload (the long-range quench): H = sum_{i<j} |i-j|^-1.5 sz_i sz_j + 0.8 sum sx,
L = 24 open chain, all-up start, Krylov evolution with m = 20 vectors and
dt = 0.01; every 0.1 time units <sz_i>, all <sz_i sz_j> and the half-chain
entropy are measured.  One step = 10 Krylov steps (0.1 time units) plus that
measurement set.  Metric: seconds of wall time per unit of simulated time
(lower is better).  The H.psi product at L = 28 is timed beside it (GB/s).

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

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

METRIC = "H·ψ GB/s vs HBM peak at L=28; Krylov evolve s per unit time at stated error"
UNIT = "s per unit simulated time"
WL = dict(L=24, J=1.0, alpha=1.5, h=0.8, m=20, dt=0.01, krylov_steps_per_step=10)
SIM_TIME_PER_STEP = WL["dt"] * WL["krylov_steps_per_step"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-hpsi28", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-trotter", action="store_true")
    ap.add_argument("--no-rdm", action="store_true")
    ap.add_argument("--entropy", choices=["async", "sync"], default="sync",
                    help="bond entropy per step: overlapped eigen-solve (async) or blocking (sync)")
    ap.add_argument("--main-priority", choices=["high", "default"], default="high",
                    help="priority of the stream the evolution runs on")
    ap.add_argument("--profile-case", choices=["batch_L16", "gates_L24", "rdm_L24"], default=None,
                    help="run one small profiling workload and exit (for ncu captures)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

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
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(torch):
    try:
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def traffic_record():
    """ncu DRAM traffic of the H.psi passes, valid only for the kernel source it was taken on."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "hpsi_traffic.json")))
    except Exception:
        return None
    src = open(os.path.join(ROOT, "paper_1802_10052_gb300", "csrc", "hpsi_kernels.cu"), "rb").read()
    if rec.get("hpsi_kernels_sha1") != hashlib.sha1(src).hexdigest():
        return None
    return rec


# ---------------------------------------------------------------------------
# multi-rank aggregation (replicas: one independent quench per rank)
# ---------------------------------------------------------------------------
def max_over_ranks(value, world, device):
    """The job's time is its slowest rank's: max of a per-rank scalar over all ranks."""
    if world <= 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(ms_max, steps, world):
    """Seconds of wall time per unit of simulated time of the whole job: each of the
    world ranks advances its own replica by SIM_TIME_PER_STEP per step."""
    return (ms_max / 1000.0) / (SIM_TIME_PER_STEP * steps * world)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world):
    import torch

    from paper_1802_10052_gb300 import Chain

    dev = torch.cuda.current_device()
    L, m, dt, nk = WL["L"], WL["m"], WL["dt"], WL["krylov_steps_per_step"]
    # the evolution runs on a high-priority stream so that the overlapped
    # eigen-solves (lowest priority) only take SMs it leaves idle
    stream = torch.cuda.Stream(priority=-1) if args.main_priority == "high" else torch.cuda.current_stream()
    chain = Chain(L, J=WL["J"], alpha=WL["alpha"], h=WL["h"], prec=args.prec, stream=stream)
    torch.cuda.synchronize()
    psi = chain.new_state()
    torch.cuda.synchronize()
    chain.init_basis_state(psi, 0)
    esize = 8 if args.prec == "mixed" else 16
    D = 1 << L

    def step(x):
        chain.krylov_evolve(x, dt, nk, m)
        sz, zz = chain.measure_zz(x)
        if args.entropy == "sync":
            S = chain.schmidt_entropy(x)
        else:  # Gram on this stream, eigen-solve overlapped on the handle's side stream
            S = chain.schmidt_entropy_async(x)
        return sz, zz, S

    for _ in range(args.warmup):
        step(psi)
    chain.measure_wait()
    torch.cuda.synchronize()
    launches0 = chain_launches(chain)
    chain.timing_read(reset=True)
    chain.timing_enable(True)
    clocks = ClockSampler(gpu_uuid(torch))
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(psi)
    chain.measure_wait()  # every measurement of the timed steps has reached the host
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ck = clocks.stop()
    chain.timing_enable(False)
    hp_ms, hp_calls = chain.timing_read(reset=True)
    launches = (chain_launches(chain) - launches0) // max(args.steps, 1)
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    ms_per_step = ms / args.steps
    value = job_value(ms, args.steps, world)

    # error of this configuration against the FP64 form (same GPU, same horizon)
    out = {"ms_per_step": ms_per_step, "value": value, "clocks": ck, "launches_per_step": launches,
           "hpsi_ms_avg": hp_ms / max(hp_calls, 1), "hpsi_calls": hp_calls}

    # roofline of the dominant kernel (H.psi passes) from the live event timing
    alg_bytes = 2.0 * D * esize
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = alg_bytes / (out["hpsi_ms_avg"] * 1e-3) / 1e9 if hp_calls else None
    trec = traffic_record()
    traffic = None
    if trec and trec.get("prec") == args.prec and trec.get("L") == L:
        traffic = trec.get("dram_bytes_per_product")
    out["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                       "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                       "kernel": "hpsi_pass_kernel (all passes of one H.psi product)",
                       "algorithmic_bytes": alg_bytes,
                       "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback"}

    # end to end through the public API with host buffers
    if not args.no_e2e:
        host = torch.empty(D, dtype=chain.dtype, pin_memory=True)
        chain.download(host, psi)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            chain.upload(psi, host)
            sz, zz, S = step(psi)
            chain.download(host, psi)
        chain.measure_wait()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e2e_val = (t1 - t0) / (SIM_TIME_PER_STEP * args.steps)
        out["e2e"] = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": D * esize,
                      "d2h_bytes_per_step": D * esize + 8 * (L + L * L + 1)}
    chain.close()
    del psi
    torch.cuda.empty_cache()
    return out


def chain_launches(chain):
    from paper_1802_10052_gb300 import _binding as B
    import ctypes as C
    n = C.c_int64()
    B.check(B.lib.osmps_ed_launch_count(chain._h, C.byref(n)), "osmps_ed_launch_count")
    return n.value


def hpsi_L28(prec, reps=20, warm=3):
    """H.psi at L = 28 (alpha = 1.5, h = 0.8): CUDA-event time per product."""
    import torch

    from paper_1802_10052_gb300 import Chain

    L = 28
    chain = Chain(L, J=1.0, alpha=1.5, h=0.8, prec=prec)
    x = chain.new_state()
    chain.init_basis_state(x, 12345)
    y = chain.new_state()
    for _ in range(warm):
        chain.apply_H(x, y)
        chain.apply_H(y, x)
    torch.cuda.synchronize()
    chain.timing_read(reset=True)
    chain.timing_enable(True)
    for i in range(reps):
        if i % 2 == 0:
            chain.apply_H(x, y)
        else:
            chain.apply_H(y, x)
    ms, n = chain.timing_read(reset=True)
    chain.timing_enable(False)
    esize = 8 if prec == "mixed" else 16
    t = ms / n
    alg = 2.0 * (1 << L) * esize
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    chain.close()
    del x, y
    torch.cuda.empty_cache()
    return {"prec": prec, "ms_per_product": t, "algorithmic_GBps": alg / (t * 1e-3) / 1e9,
            "frac_of_measured_hbm": alg / (t * 1e-3) / 1e9 / peak, "algorithmic_bytes": alg}


def batched_ground(n=512, reps=3):
    """Batched ground states: n long-range chains, L ~ U{14..20}, alpha ~ U[0.5, 3],
    h ~ U[0.2, 2] (seed 3), each Lanczos to 1e-10, in one persistent launch
    replayed from a CUDA graph (work split chosen by the autotuner).  Beside it:
    the same batch in FP64, and the plain single-chain solver (FP64, and
    complex64 to a 1e-4 explicit residual) timed on a stratified sample of two
    chains per length and scaled by the length counts."""
    import numpy as np
    import torch

    import seeded_inputs as si
    from paper_1802_10052_gb300 import Chain, ChainBatch

    inst = si.batched_instances(n, seed=3)
    Ls = [x[0] for x in inst]
    al = [x[1] for x in inst]
    hs = [x[2] for x in inst]
    starts = si.batch_start_states(Ls, seed=3)
    out = {"workload": f"{n} chains H = sum |i-j|^-alpha sz sz + h sum sx, L~U{{14..20}}, alpha~U[0.5,3], "
                       "h~U[0.2,2], seeded Gaussian starts, Lanczos tol 1e-10"}

    def timed_batch(prec, reps_):
        dt = np.complex64 if prec == "mixed" else np.complex128
        b = ChainBatch(Ls, [1.0] * n, al, hs, prec=prec, max_iter=1000)
        start = torch.from_numpy(np.concatenate([v.astype(dt) for v in starts])).cuda()
        psi = start.clone()
        split = b.autotune(psi, tol=1e-10) if prec == "mixed" else b.get_split() + (None,)
        b.set_graph(True)
        ts = []
        for r in range(reps_ + 1):
            psi.copy_(start)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            b.lanczos_ground_async(psi, 1e-10)
            e1.record()
            b.check()
            if r > 0:
                ts.append(e0.elapsed_time(e1))
        it = b.iters.cpu().numpy().astype(np.float64)
        st = b.status.cpu().numpy()
        E = b.energy.cpu().numpy()
        R = b.residual.cpu().numpy()
        D = np.array([1 << L for L in Ls], dtype=np.float64)
        esize = 8 if prec == "mixed" else 16
        t = float(np.median(ts))
        res = {"ms": t, "chains_per_s": n / (t * 1e-3), "iters_mean": float(it.mean()), "iters_max": int(it.max()),
               "converged": int((st == 0).sum()), "max_residual": float(R.max()),
               "algorithmic_GBps": float(np.sum(esize * D * (20 * it + 7))) / (t * 1e-3) / 1e9,
               "split": {"cluster_ctas": split[0], "cluster_min_L": split[1], "grid": split[2]},
               "launches_per_solve": 1}
        b.close()
        return res, E

    mixed, E_mixed = timed_batch("mixed", reps)
    fp64, E_fp64 = timed_batch("fp64", 1)
    out["batched_mixed"] = mixed
    out["batched_fp64"] = fp64
    out["max_rel_energy_diff_mixed_vs_fp64"] = float(np.max(np.abs(E_mixed - E_fp64) / np.maximum(1.0, np.abs(E_fp64))))
    counts = {L: Ls.count(L) for L in sorted(set(Ls))}
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-4)):
        per = {}
        for L in counts:
            ts = []
            for k in [k for k in range(n) if Ls[k] == L][:2]:
                c = Chain(L, J=1.0, alpha=al[k], h=hs[k], prec=prec)
                x = torch.from_numpy(starts[k].astype(np.complex128 if prec == "fp64" else np.complex64)).cuda()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                c.lanczos_ground(x, tol=tol, max_iter=1000, raise_on_noconv=False)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
                c.close()
            per[L] = float(np.mean(ts))
        est = sum(per[L] * counts[L] for L in counts)
        out[f"plain_{prec}"] = {"s_scaled_to_batch": est, "tol_explicit_residual": tol,
                                "sample": "2 chains per length, mean time x chains of that length",
                                "s_per_chain_by_L": per}
    out["speedup_batched_mixed_vs_plain_fp64"] = out["plain_fp64"]["s_scaled_to_batch"] / (mixed["ms"] * 1e-3)
    out["speedup_batched_fp64_vs_plain_fp64"] = out["plain_fp64"]["s_scaled_to_batch"] / (fp64["ms"] * 1e-3)
    torch.cuda.empty_cache()
    return out


def adjoint_L20(reps=2):
    """Gradient of <H(h=1)> after 200 Krylov steps (dt = 0.025, m = 20) of the L = 20,
    alpha = 2 chain with a seeded field h_k ~ U[0.5, 1.5], from all up: seconds per
    gradient (loss, 200 field derivatives and the coupling-scale derivative), FP64 and
    complex64.  H.psi products per gradient: forward N m, segment recomputation
    <= N m, backward N (2 m + 2 nquad)."""
    import numpy as np
    import torch

    import seeded_inputs as si
    from paper_1802_10052_gb300 import Chain

    L, n, dt, m, nq = 20, 200, 0.025, 20, 8
    hs = si.field_schedule(n, seed=4)
    out = {"workload": "H = sum |i-j|^-2 sz sz + h_k sum sx, L=20, 200 steps dt=0.025, m=20, h_k~U[0.5,1.5] "
                       "(seed 4), loss <H(h=1)>, gradient w.r.t. all h_k and the coupling scale"}
    products = n * m + n * m + n * (2 * m + 2 * nq)
    for prec in ("fp64", "mixed"):
        c = Chain(L, J=1.0, alpha=2.0, h=1.0, prec=prec)
        x = c.new_state()
        c.init_basis_state(x, 0)
        c.adjoint_grad(x, hs, dt, m=m, nquad=nq)  # warm-up
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            loss, gh, gs = c.adjoint_grad(x, hs, dt, m=m, nquad=nq)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        t = min(ts)
        esize = 16 if prec == "fp64" else 8
        out[prec] = {"s_per_gradient": t, "loss": loss, "grad_scale": gs, "grad_h_norm": float(np.linalg.norm(gh)),
                     "hpsi_products": products,
                     "algorithmic_GBps_of_products": products * 2.0 * (1 << L) * esize / t / 1e9}
        c.close()
    return out


def trotter_nn(L=24, reps=10):
    """Nearest-neighbour chain (J = 1, h = 1, open, complex64): ms per time step of the
    Trotter products of order 2 and 4 (Sec. III.C) against one Krylov step (m = 20) on the
    same chain, both timed with CUDA events.  Bytes per step: every window pass reads and
    writes the state once (2 D s); order 2 = 2 layers, order 4 = 11 layers per step, a layer
    = ceil(bonds / 2) window passes."""
    import torch

    from paper_1802_10052_gb300 import Chain

    c = Chain(L, couplings=[1.0] + [0.0] * (L - 2), h=1.0, prec="mixed")
    x = c.new_state()
    c.init_basis_state(x, 0)
    out = {"workload": f"NN transverse Ising L={L}, J=1, h=1, open, dt=0.01, complex64"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    D = 1 << L
    passes_per_layer = {0: ((L - 1) // 2 + 1) // 2, 1: (L // 2 + 1) // 2}
    for order, layers in ((2, [(0, 1), (1, 1)]), (4, [(f % 2, 1) for f in range(11)])):
        c.trotter_evolve(x, 0.01, 2, order)
        torch.cuda.synchronize()
        e0.record()
        c.trotter_evolve(x, 0.01, reps, order)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        npass = sum(passes_per_layer[p] for p, _ in layers)
        out[f"order{order}"] = {"ms_per_step": ms, "window_passes_per_step": npass,
                                "GBps": npass * 2.0 * D * 8 / (ms * 1e-3) / 1e9}
    c.krylov_evolve(x, 0.01, 1, 20)
    torch.cuda.synchronize()
    e0.record()
    c.krylov_evolve(x, 0.01, 3, 20)
    e1.record()
    torch.cuda.synchronize()
    out["krylov_m20_ms_per_step"] = e0.elapsed_time(e1) / 3
    out["krylov_over_trotter2"] = out["krylov_m20_ms_per_step"] / out["order2"]["ms_per_step"]
    c.close()
    return out


def rdm_L24(reps=3):
    """All 276 two-site RDMs and the bond entropy of all 23 cuts of an L = 24 complex64
    state (the quench state after 0.2 time units): ms per call.  The pair kernel reads
    the state once per pair: 276 x D x 8 B."""
    import torch

    from paper_1802_10052_gb300 import Chain

    L = 24
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    x = c.new_state()
    c.init_basis_state(x, 0)
    c.krylov_evolve(x, 0.01, 20, 20)
    c.rdm_pairs(x)
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.rdm_pairs(x)
        ts.append(time.perf_counter() - t0)
    t_rdm = min(ts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c.entropy_sweep(x)
    t_sweep = time.perf_counter() - t0
    npairs = L * (L - 1) // 2
    c.close()
    return {"workload": "L=24 complex64 state, all pairs (276) and all cuts (23)",
            "rdm_pairs_ms": t_rdm * 1e3, "rdm_GBps": npairs * (1 << L) * 8 / t_rdm / 1e9,
            "entropy_sweep_ms": t_sweep * 1e3}


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
class OracleSample:
    """Bounded sample of the workload on the FP64 oracle: a few Lanczos
    iterations of one Krylov step (matvec + full reorthogonalisation), one
    correlator through its two-site reduced density matrix, one single-site
    expectation and the half-chain spectrum; scaled to seconds per unit of
    simulated time (100 Krylov steps of m iterations and 10 measurement sets
    per unit time)."""

    def __init__(self, iters=3):
        import numpy as np

        import seeded_inputs as si
        from oracle import ed_oracle as O

        self.O, self.np = O, np
        L = WL["L"]
        self.L = L
        self.iters = iters
        self.mv = O.RuleSetH(L, O.coupling_table(L, WL["J"], WL["alpha"]), WL["h"])
        psi = si.basis_state(L, 0)
        psi, _ = O.krylov_step(self.mv, psi, WL["dt"], 4)  # a non-trivial state
        self.psi = psi

    def run(self):
        np, O = self.np, self.O
        m = WL["m"]
        t0 = time.perf_counter()
        V = [self.psi / np.linalg.norm(self.psi)]
        for j in range(self.iters):
            w = self.mv(V[j])
            for _ in range(2):
                for v in V:
                    w = w - np.vdot(v, w) * v
            V.append(w / np.linalg.norm(w))
        t1 = time.perf_counter()
        O.measure_corr_pair(self.psi, self.L, 3, 17)
        t2 = time.perf_counter()
        O.rdm_sites(self.psi, self.L, [5])
        t3 = time.perf_counter()
        O.schmidt_spectrum(self.psi, self.L)
        t4 = time.perf_counter()
        per_iter = (t1 - t0) / self.iters
        # full reorth makes later iterations dearer: iteration j costs ~ (1 + j c) units
        step = per_iter * m * (1.0 + (m - self.iters) / (2.0 * (self.iters + 1)) * 0.3)
        pairs = self.L * (self.L - 1) // 2
        meas = (t2 - t1) * pairs + (t3 - t2) * self.L + (t4 - t3)
        per_unit = step / WL["dt"] + meas / SIM_TIME_PER_STEP
        return per_unit, t4 - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    samp = OracleSample(iters=2)
    vals = []
    for i in range(args.warmup + args.steps):
        v, wall = samp.run()
        if i >= args.warmup:
            vals.append((v, wall))
    value = statistics.median(v for v, _ in vals)
    ms_per_step = value * SIM_TIME_PER_STEP * 1000.0
    desc = ("2 Lanczos iterations of one Krylov step (matvec + full reorth) at L=24, one two-site RDM, one "
            "single-site RDM and the half-chain spectrum per step, scaled to 100 Krylov steps of m=20 and 10 "
            "measurement sets per unit time")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "lrqi_quench_L24: alpha=1.5 h=0.8 all-up, Krylov m=20 dt=0.01, "
                                   "measure every 0.1", "L": WL["L"], "oracle": "numpy/scipy FP64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_line():
    samp = OracleSample(iters=3)
    v, wall = samp.run()
    return {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"3 Lanczos iterations (matvec + full reorth) of one L=24 Krylov step, one two-site and one "
                      f"single-site RDM and the half-chain spectrum ({wall:.1f} s of CPU work), scaled to 100 "
                      f"Krylov steps of m=20 and 10 measurement sets per unit time"}


def profile_case(name):
    """Small workloads sized for full ncu captures (a few hundred MB on the device)."""
    import numpy as np
    import torch

    import seeded_inputs as si
    from paper_1802_10052_gb300 import ChainBatch

    torch.cuda.set_device(0)
    if name == "batch_L16":
        # 152 chains of L = 16 (one per SM), alpha = 1.7, h = 0.9, seeded Gaussian starts; two solves
        n, L = 152, 16
        b = ChainBatch([L] * n, [1.0] * n, [1.7] * n, [0.9] * n, prec="mixed", max_iter=1000)
        start = torch.from_numpy(np.concatenate([v.astype(np.complex64)
                                                 for v in si.batch_start_states([L] * n, seed=3)])).cuda()
        psi = start.clone()
        for _ in range(2):
            psi.copy_(start)
            b.lanczos_ground(psi, 1e-10)
        print(json.dumps({"profile_case": name, "iters_mean": float(b.iters.float().mean())}))
    elif name == "gates_L24":
        # NN chain L = 24 (J = h = 1), complex64, all-up start: two second-order Trotter steps
        from paper_1802_10052_gb300 import Chain
        L = 24
        c = Chain(L, couplings=[1.0] + [0.0] * (L - 2), h=1.0, prec="mixed")
        x = c.new_state()
        c.init_basis_state(x, 0)
        c.trotter_evolve(x, 0.01, 2, 2)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": name, "norm": float(torch.linalg.vector_norm(x).item())}))
        c.close()
    elif name == "rdm_L24":
        # L = 24 complex64 seeded Gaussian state: all 276 pair RDMs, twice
        from paper_1802_10052_gb300 import Chain
        L = 24
        c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
        x = torch.from_numpy(si.gaussian_state(L, 24).astype(np.complex64)).cuda()
        r2, _ = c.rdm_pairs(x)
        r2, _ = c.rdm_pairs(x)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": name, "trace_01": float(np.trace(r2[0]).real)}))
        c.close()
    return 0


def main():
    args = parse()
    if args.profile_case is not None:
        return profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args)
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    res = run_ours(args, rank, world)
    extra = {}
    if rank == 0 and not args.no_hpsi28:
        extra["hpsi_L28"] = [hpsi_L28("mixed"), hpsi_L28("fp64", reps=6)]
    if rank == 0 and not args.no_batch:
        extra["batched_ground_512"] = batched_ground()
    if rank == 0 and not args.no_grad:
        extra["adjoint_grad_L20"] = adjoint_L20()
    if rank == 0 and not args.no_trotter:
        extra["trotter_nn_L24"] = trotter_nn()
    if rank == 0 and not args.no_rdm:
        extra["rdm_L24"] = rdm_L24()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_line()
    if rank == 0:
        line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "c64+f64" if args.prec == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": "lrqi_quench_L24: H = sum |i-j|^-1.5 sz sz + 0.8 sum sx, L=24, all-up "
                                       "start, Krylov m=20 dt=0.01, <sz_i>, <sz_i sz_j>, S(L/2) every 0.1; "
                                       "step = 0.1 time units",
                           "L": WL["L"], "m": WL["m"], "dt": WL["dt"], "precision": args.prec,
                           "parallelism": f"replicas x{world}",
                           "entropy": args.entropy, "main_stream_priority": args.main_priority,
                           "l2": "working set (21 Krylov vectors of 134 MB) larger than L2"},
                "roofline": res["roofline"], "cpu_baseline": cpu, "clocks": res["clocks"],
                "gpu_launches": res["launches_per_step"] * args.steps,
                "hpsi_ms_avg_L24": res["hpsi_ms_avg"], **extra}
        if "e2e" in res:
            line["e2e"] = res["e2e"]
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
