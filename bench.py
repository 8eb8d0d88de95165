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
    ap.add_argument("--no-fp64-arm", action="store_true")
    ap.add_argument("--no-scale", action="store_true")
    ap.add_argument("--no-entropy-routes", action="store_true")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--entropy", choices=["async", "sync"], default="sync",
                    help="bond entropy per step: overlapped eigen-solve (async) or blocking (sync)")
    ap.add_argument("--main-priority", choices=["high", "default"], default="high",
                    help="priority of the stream the evolution runs on")
    ap.add_argument("--profile-case", choices=["batch_L16", "gates_L24", "rdm_L24", "hpsi_L27", "quench_L24",
                                               "hpsi_fp64_L24", "krylov_L24", "entropy_L24"],
                    default=None,
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


def traffic_record(L, prec):
    """ncu DRAM traffic of one H.psi product at size L, valid only for the kernel source it was taken on."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "hpsi_traffic.json")))
    except Exception:
        return None
    src = open(os.path.join(ROOT, "paper_1802_10052_gb300", "csrc", "hpsi_kernels.cu"), "rb").read()
    if rec.get("hpsi_kernels_sha1") != hashlib.sha1(src).hexdigest():
        return None
    for r in rec.get("records", []):
        if r.get("L") == L and r.get("prec") == prec:
            return r
    return None


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
def energy_all_up(L, J, alpha):
    """<up|H|up> = sum_r (L - r) J(r): conserved by the exact evolution from all up."""
    return sum((L - r) * J / r ** alpha for r in range(1, L))


def run_arm(args, prec, steps, warmup, world, e2e=True):
    """The quench at L = 24 in one precision: `warmup` untimed steps, then `steps`
    steps timed with CUDA events on the evolution's stream.  Every step's
    measurements are kept (the trajectory of t = 0.1, 0.2, ...) so that the two
    precisions can be compared point by point."""
    import numpy as np
    import torch

    from paper_1802_10052_gb300 import Chain

    L, m, dt, nk = WL["L"], WL["m"], WL["dt"], WL["krylov_steps_per_step"]
    # the evolution runs on a high-priority stream so that the overlapped
    # eigen-solves (lowest priority) only take SMs it leaves idle
    stream = torch.cuda.Stream(priority=-1) if args.main_priority == "high" else torch.cuda.current_stream()
    chain = Chain(L, J=WL["J"], alpha=WL["alpha"], h=WL["h"], prec=prec, stream=stream)
    torch.cuda.synchronize()
    psi = chain.new_state()
    torch.cuda.synchronize()
    chain.init_basis_state(psi, 0)
    esize = 8 if prec == "mixed" else 16
    D = 1 << L
    traj = []
    err_est = [0.0]

    def step(x):
        err_est[0] += chain.krylov_evolve(x, dt, nk, m)
        sz, zz = chain.measure_zz(x)
        if args.entropy == "sync":
            S = chain.schmidt_entropy(x)
        else:  # Gram on this stream, eigen-solve overlapped on the handle's side stream
            S = chain.schmidt_entropy_async(x)
        return sz, zz, S

    def keep(out):
        sz, zz, S = out
        traj.append((sz, zz, S))

    for _ in range(warmup):
        keep(step(psi))
    chain.measure_wait()
    torch.cuda.synchronize()
    if e2e:
        # the state where the timed steps start: the end-to-end leg repeats the same
        # stretch of the trajectory (the cost of a measurement depends on how many
        # Schmidt values matter, which grows along it)
        host_start = torch.empty(D, dtype=chain.dtype, pin_memory=True)
        chain.download(host_start, psi)
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
    for _ in range(steps):
        keep(step(psi))
    chain.measure_wait()  # every measurement of the timed steps has reached the host
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ck = clocks.stop()
    chain.timing_enable(False)
    hp_ms, hp_calls = chain.timing_read(reset=True)
    launches = (chain_launches(chain) - launches0) // max(steps, 1)
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    traj = [(np.asarray(a), np.asarray(b), float(c.S if hasattr(c, "S") else c)) for a, b, c in traj]
    E, n2 = chain.energy(psi)
    out = {"ms": ms, "ms_per_step": ms / steps, "value": job_value(ms, steps, world), "clocks": ck,
           "launches_per_step": launches, "hpsi_ms_avg": hp_ms / max(hp_calls, 1), "hpsi_calls": hp_calls,
           "traj": traj, "energy": E, "norm2": n2, "krylov_err_estimate": err_est[0],
           "t_end": (warmup + steps) * SIM_TIME_PER_STEP, "psi_final": psi.cpu()}
    # end to end through the public API with host buffers
    if e2e:
        host = host_start
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            chain.upload(psi, host)
            sz, zz, S = step(psi)
            chain.download(host, psi)
        chain.measure_wait()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        out["e2e"] = {"value": (t1 - t0) / (SIM_TIME_PER_STEP * steps), "unit": UNIT,
                      "h2d_bytes_per_step": D * esize, "d2h_bytes_per_step": D * esize + 8 * (L + L * L + 1)}
    chain.close()
    del psi
    torch.cuda.empty_cache()
    return out


def arm_errors(mixed, fp64):
    """Sec. V error measures of the complex64 run against the FP64 run of the same
    quench, point by point along the common trajectory, plus the final states."""
    import numpy as np

    n = min(len(mixed["traj"]), len(fp64["traj"]))
    dsz = max(float(np.max(np.abs(a[0] - b[0]))) for a, b in zip(mixed["traj"][:n], fp64["traj"][:n]))
    dzz = max(float(np.max(np.abs(a[1] - b[1]))) for a, b in zip(mixed["traj"][:n], fp64["traj"][:n]))
    dS = max(abs(a[2] - b[2]) for a, b in zip(mixed["traj"][:n], fp64["traj"][:n]))
    pm = mixed["psi_final"].numpy().astype(np.complex128)
    pf = fp64["psi_final"].numpy()
    same_t = abs(mixed["t_end"] - fp64["t_end"]) < 1e-12
    return {"points": n, "t_max": n * SIM_TIME_PER_STEP, "max_abs_sz": dsz, "max_abs_szsz": dzz, "max_abs_S": dS,
            "final_state_rel_l2": float(np.linalg.norm(pm - pf) / np.linalg.norm(pf)) if same_t else None,
            "final_energy_rel": abs(mixed["energy"] - fp64["energy"]) / abs(fp64["energy"]) if same_t else None,
            "tolerance": 1e-5, "within_tolerance": bool(max(dsz, dzz, dS) <= 1e-5)}


def conservation(arm, E0):
    """Errors against what the exact evolution fixes: <psi|psi> = 1 and <H> = E0."""
    return {"t": arm["t_end"], "energy_rel_err": abs(arm["energy"] / arm["norm2"] - E0) / abs(E0),
            "norm_err": abs(arm["norm2"] - 1.0), "krylov_err_estimate": arm["krylov_err_estimate"]}


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


def scale_L30():
    """The scale workload: H = sum |i-j|^-1 sz sz + 1.2 sum sx, L = 30, complex64, Krylov
    dimension 12, from the Neel state to t = 2 in 100 steps of 0.02 (seconds per unit of
    simulated time, CUDA events), the H.psi product at L = 30 (GB/s), and the half-chain
    spectrum at t = 2 through the tensor-core Gram product of 32768 x 32768 and its
    eigenvalues; unitarity and energy conservation at t = 2."""
    import torch

    import seeded_inputs as si
    from paper_1802_10052_gb300 import Chain

    L, alpha, h, dt, m, n = 30, 1.0, 1.2, 0.02, 12, 100
    c = Chain(L, J=1.0, alpha=alpha, h=h, prec="mixed")
    x = c.new_state()
    c.init_basis_state(x, si.neel_index(L))
    e0 = sum((L - r) * (-1) ** r / r ** alpha for r in range(1, L))
    torch.cuda.synchronize()
    c.timing_read(reset=True)
    c.timing_enable(True)
    e_0, e_1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_0.record()
    c.krylov_evolve(x, dt, n, m)
    e_1.record()
    torch.cuda.synchronize()
    hp_ms, hp_n = c.timing_read(reset=True)
    c.timing_enable(False)
    ms = e_0.elapsed_time(e_1)
    E, n2 = c.energy(x)
    t0 = time.perf_counter()
    S, lam = c.schmidt_entropy(x, spectrum=True)
    t_ent = time.perf_counter() - t0
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    alg = 2.0 * (1 << L) * 8
    t_hp = hp_ms / max(hp_n, 1)
    out = {"workload": "H = sum |i-j|^-1 sz sz + 1.2 sum sx, L=30, complex64, Neel start, Krylov m=12, "
                       "100 steps of dt=0.02 to t=2",
           "s_per_unit_time": ms * 1e-3 / (n * dt), "hpsi_ms_per_product": t_hp,
           "hpsi_algorithmic_GBps": alg / (t_hp * 1e-3) / 1e9, "hpsi_frac_of_measured_hbm": alg / (t_hp * 1e-3) / 1e9 / peak,
           "entropy_s": t_ent, "entropy_route": "tensor-core Gram 32768 x 32768 + eigenvalues", "S_t2": S,
           "lambda0_t2": float(lam[0]), "norm_err_t2": abs(n2 - 1.0), "energy_rel_err_t2": abs(E / n2 - e0) / abs(e0)}
    c.close()
    del x
    torch.cuda.empty_cache()
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


def entropy_routes_L24(times=(0.5, 1.0, 2.5)):
    """Half-chain entropy of the L = 24 quench state (complex64) at a few times: ms per
    measurement on the dominant subspace (method 4, the default; second call on the
    handle, so it starts from the dimension the first found) and on the full route
    (Gram eigenvectors, Rayleigh quotients; method 2), and |dS| between them."""
    import numpy as np
    import torch

    from paper_1802_10052_gb300 import Chain

    c = Chain(24, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    x = c.new_state()
    c.init_basis_state(x, 0)
    t = 0.0
    out = {"workload": "L=24 quench state (alpha=1.5, h=0.8, all up, Krylov m=20 dt=0.01), complex64, cut 12|12",
           "points": []}

    def timed(method):
        c.set_entropy_method(method)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S, lam = c.schmidt_entropy(x, spectrum=True)
        return S, lam, (time.perf_counter() - t0) * 1e3

    for target in times:
        steps = int(round((target - t) / 0.01))
        c.krylov_evolve(x, 0.01, steps, 20)
        t = target
        timed(4)
        S4, lam4, ms4 = timed(4)
        timed(2)  # the library solver's first call sets itself up
        S2, lam2, ms2 = timed(2)
        out["points"].append({"t": t, "subspace_ms": ms4, "full_ms": ms2, "S": S4, "abs_dS": abs(S4 - S2),
                              "values_above_1e-12": int(np.sum(lam4 > 1e-12))})
    c.close()
    return out


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
class OracleSample:
    """Bounded sample of the workload on the FP64 oracle, scaled to seconds per
    unit of simulated time by exact operation counts.

    The oracle's Krylov step (krylov_step, m = 20, basis orthogonalised twice
    against all previous vectors) performs per step: m rule-set products,
    m + 2 sum_{j<m}(j+1) inner products, m + (m-1) + 2 sum_{j<m}(j+1) + m vector
    updates (w - c v and the combination), m + 1 norms and m scalings of a
    2^24-amplitude state.  A measurement set is L single-site and L(L-1)/2 pair
    reduced density matrices and one half-chain spectrum.  Every unit is timed
    here on the workload's own state: one product, a few inner products,
    updates, norms and scalings (the same numpy expressions krylov_step
    evaluates), one single-site and one pair density matrix, and (once) the
    spectrum.  The rule set's one-time setup (the diagonal by the pair loop) is
    amortised over the workload's whole run to t = 5."""

    T_RUN = 5.0

    def __init__(self):
        import numpy as np

        import seeded_inputs as si
        from oracle import ed_oracle as O

        self.O, self.np = O, np
        L = WL["L"]
        self.L = L
        t0 = time.perf_counter()
        self.mv = O.RuleSetH(L, O.coupling_table(L, WL["J"], WL["alpha"]), WL["h"])
        self.t_setup = time.perf_counter() - t0
        psi = si.basis_state(L, 0)
        psi, _ = O.krylov_step(self.mv, psi, WL["dt"], 2)  # a non-trivial state
        self.psi = psi
        t0 = time.perf_counter()
        O.schmidt_spectrum(psi, L)
        self.t_spec = time.perf_counter() - t0

    def counts(self):
        m = WL["m"]
        tri = m * (m + 1) // 2
        return {"matvec": m, "vdot": m + 2 * tri, "axpy": m + (m - 1) + 2 * tri + m, "norm": m + 1, "scale": m}

    def run(self):
        """One sample; returns (seconds per unit simulated time, wall seconds of the sample)."""
        np, O = self.np, self.O
        t_start = time.perf_counter()
        w = self.mv(self.psi)
        t_mv = time.perf_counter() - t_start
        v = self.psi
        reps = 4
        t0 = time.perf_counter()
        for _ in range(reps):
            c = np.vdot(v, w)
        t_vdot = (time.perf_counter() - t0) / reps
        t0 = time.perf_counter()
        for _ in range(reps):
            u = w - c * v
        t_axpy = (time.perf_counter() - t0) / reps
        t0 = time.perf_counter()
        for _ in range(reps):
            b = float(np.linalg.norm(u))
        t_norm = (time.perf_counter() - t0) / reps
        t0 = time.perf_counter()
        for _ in range(reps):
            _ = u / b
        t_scale = (time.perf_counter() - t0) / reps
        t0 = time.perf_counter()
        O.measure_corr_pair(self.psi, self.L, 3, 17)
        t_pair = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.rdm_sites(self.psi, self.L, [5])
        t_site = time.perf_counter() - t0
        wall = time.perf_counter() - t_start
        n = self.counts()
        step = (n["matvec"] * t_mv + n["vdot"] * t_vdot + n["axpy"] * t_axpy + n["norm"] * t_norm
                + n["scale"] * t_scale)
        pairs = self.L * (self.L - 1) // 2
        meas = pairs * t_pair + self.L * t_site + self.t_spec
        per_unit = step / WL["dt"] + meas / SIM_TIME_PER_STEP + self.t_setup / self.T_RUN
        self.last = {"krylov_step_s": step, "measurement_set_s": meas, "matvec_s": t_mv, "vdot_s": t_vdot,
                     "axpy_s": t_axpy, "pair_rdm_s": t_pair, "site_rdm_s": t_site, "spectrum_s": self.t_spec,
                     "setup_s": self.t_setup}
        return per_unit, wall

    def describe(self):
        return ("unit costs timed on the L=24 quench state (one rule-set product, numpy inner products, updates, "
                "norms and scalings of 2^24 amplitudes, one pair and one single-site RDM, the half-chain spectrum), "
                "scaled by the exact operation counts of the oracle's Krylov step (m=20, two Gram-Schmidt passes) "
                "x 100 steps and 10 measurement sets (276 pair RDMs, 24 site RDMs, 1 spectrum) per unit time, plus "
                f"the rule set's setup ({self.t_setup:.0f} s) over a run to t=5")


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


ONE_THREAD = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def run_reference(args):
    """The FP64 oracle timed on the host (rank 0 only), one thread for BLAS as
    for the elementwise numpy work (the paper's own code ran on one core)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    samp = OracleSample()
    vals, walls = [], []
    for i in range(args.warmup + args.steps):
        v, wall = samp.run()
        if i >= args.warmup:
            vals.append(v)
            walls.append(wall)
    value = statistics.median(vals)
    cores = 1 if os.environ.get("OMP_NUM_THREADS") == "1" else cpu_cores()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.median(walls), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "lrqi_quench_L24: alpha=1.5 h=0.8 all-up, Krylov m=20 dt=0.01, "
                                   "measure every 0.1", "L": WL["L"], "oracle": "numpy/scipy FP64",
                       "ms_per_step": "wall time of one bounded sample; value = that sample scaled to the workload"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": samp.describe(),
                             "cpu_model": cpu_model(), "host_cores": cpu_cores(), "units": samp.last},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def oracle_sample_main():
    """`--oracle-sample`: one bounded sample printed as JSON (run in a child
    process so that its thread count is fixed before numpy loads)."""
    samp = OracleSample()
    v, wall = samp.run()
    print(json.dumps({"value": v, "wall_s": wall, "units": samp.last, "sample": samp.describe()}), flush=True)
    return 0


def cpu_baseline_line():
    env = dict(os.environ, **ONE_THREAD)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample"], capture_output=True, text=True,
                       env=env, timeout=1200)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: " + r.stderr[-300:]}
    res = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": res["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": res["sample"] + f" ({res['wall_s']:.1f} s of CPU work in the sample)", "cpu_model": cpu_model(),
            "host_cores": cpu_cores(), "units": res["units"]}


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
    elif name == "hpsi_L27":
        # H.psi at L = 27 (alpha = 1.5, h = 0.8), complex64, seeded Gaussian state drawn on the
        # device: the first three-pass size; two products (3 GB on the device)
        from paper_1802_10052_gb300 import Chain
        L = 27
        c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
        g = torch.Generator(device="cuda")
        g.manual_seed(27)
        x = torch.complex(torch.randn(1 << L, generator=g, device="cuda"), torch.randn(1 << L, generator=g, device="cuda"))
        y = c.new_state()
        c.apply_H(x, y)
        c.apply_H(y, x)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": name, "norm": float(torch.linalg.vector_norm(x).item())}))
        c.close()
    elif name == "hpsi_fp64_L24":
        # complex128 H.psi at L = 24 (alpha = 1.5, h = 0.8): one product with the flip sums in
        # 64-bit fixed point, one with FP64 multiply-adds (three passes each)
        from paper_1802_10052_gb300 import Chain
        L = 24
        c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="fp64")
        x = torch.from_numpy(si.gaussian_state(L, 24)).cuda()
        y = c.new_state()
        for mode in (1, 0):
            c.set_flip_sums(mode)
            c.apply_H(x, y)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": name, "norm": float(torch.linalg.vector_norm(y).item())}))
        c.close()
    elif name == "entropy_L24":
        # the half-chain entropy of the L = 24 quench state at t = 1 (complex64, default
        # route: the dominant subspace, p = 128), three calls
        from paper_1802_10052_gb300 import Chain
        c = Chain(WL["L"], J=WL["J"], alpha=WL["alpha"], h=WL["h"], prec="mixed")
        x = c.new_state()
        c.init_basis_state(x, 0)
        c.krylov_evolve(x, WL["dt"], 100, WL["m"])
        S = [c.schmidt_entropy(x) for _ in range(3)]
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": name, "S": S}))
        c.close()
    elif name == "krylov_L24":
        # one Krylov step (m = 20) of the L = 24 quench state at t = 0.1, complex64: 20 products
        # with the Krylov epilogue, as in the benchmark step
        from paper_1802_10052_gb300 import Chain
        c = Chain(WL["L"], J=WL["J"], alpha=WL["alpha"], h=WL["h"], prec="mixed")
        x = c.new_state()
        c.init_basis_state(x, 0)
        c.krylov_evolve(x, WL["dt"], 11, WL["m"])
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": name}))
        c.close()
    elif name == "quench_L24":
        # the benchmark workload (10 Krylov steps, <sz>, <szsz>, S per step), complex64: five
        # untimed steps to t = 0.5, then two steps inside the NVTX range "step" (for ncu --nvtx)
        from paper_1802_10052_gb300 import Chain
        c = Chain(WL["L"], J=WL["J"], alpha=WL["alpha"], h=WL["h"], prec="mixed")
        x = c.new_state()
        c.init_basis_state(x, 0)
        for k in range(7):
            if k == 5:
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_push("step")
            c.krylov_evolve(x, WL["dt"], WL["krylov_steps_per_step"], WL["m"])
            c.measure_zz(x)
            S = c.schmidt_entropy(x)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_case": name, "S": S}))
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
    if args.oracle_sample:
        return oracle_sample_main()
    if args.profile_case is not None:
        return profile_case(args.profile_case)
    if args.impl == "reference":
        for k, v in ONE_THREAD.items():
            os.environ.setdefault(k, v)
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
    res = run_arm(args, args.prec, args.steps, args.warmup, world, e2e=not args.no_e2e)
    extra = {}
    E0 = energy_all_up(WL["L"], WL["J"], WL["alpha"])
    extra["conservation"] = conservation(res, E0)
    extra["hpsi_ms_avg_L24"] = res["hpsi_ms_avg"]
    if rank == 0 and not args.no_fp64_arm and args.prec == "mixed":
        f = run_arm(args, "fp64", args.steps, args.warmup, 1, e2e=False)
        extra["fp64_arm"] = {"value": f["value"], "unit": UNIT, "ms_per_step": f["ms_per_step"],
                             "hpsi_ms_avg_L24": f["hpsi_ms_avg"], "conservation": conservation(f, E0),
                             "clocks": f["clocks"],
                             "mixed_speedup": f["value"] / res["value"]}
        extra["error_vs_fp64"] = arm_errors(res, f)
        del f
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    esize = 8 if args.prec == "mixed" else 16
    D = 1 << WL["L"]
    alg24 = 2.0 * D * esize
    ach24 = alg24 / (res["hpsi_ms_avg"] * 1e-3) / 1e9 if res["hpsi_calls"] else None
    t24 = traffic_record(WL["L"], args.prec)
    extra["roofline_L24"] = {"bound": "hbm", "achieved": ach24, "peak": peak, "unit": "GB/s",
                             "frac": ach24 / peak if ach24 else None, "algorithmic_bytes": alg24,
                             "traffic": t24.get("dram_bytes_per_product") if t24 else None,
                             "kernel": "hpsi_pass_kernel (all passes of one H.psi product, in the timed step)"}
    roof = None
    if rank == 0 and not args.no_hpsi28:
        h28 = [hpsi_L28("mixed"), hpsi_L28("fp64", reps=6)]
        extra["hpsi_L28"] = h28
        r = h28[0] if args.prec == "mixed" else h28[1]
        trec = traffic_record(28, args.prec)
        traffic = trec.get("dram_bytes_per_product") if trec else None
        roof = {"bound": "hbm", "achieved": r["algorithmic_GBps"], "peak": peak, "unit": "GB/s",
                "frac": r["algorithmic_GBps"] / peak, "traffic": traffic,
                "kernel": "hpsi_pass_kernel (all passes of one H.psi product), L=28 alpha=1.5 h=0.8",
                "algorithmic_bytes": r["algorithmic_bytes"], "ms_per_product": r["ms_per_product"],
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback"}
    if rank == 0 and not args.no_batch:
        extra["batched_ground_512"] = batched_ground()
    if rank == 0 and not args.no_grad:
        extra["adjoint_grad_L20"] = adjoint_L20()
    if rank == 0 and not args.no_trotter:
        extra["trotter_nn_L24"] = trotter_nn()
    if rank == 0 and not args.no_rdm:
        extra["rdm_L24"] = rdm_L24()
    if rank == 0 and not args.no_scale:
        extra["scale_L30"] = scale_L30()
    if rank == 0 and not args.no_entropy_routes:
        try:
            extra["entropy_routes_L24"] = entropy_routes_L24()
        except Exception as e:  # a leg of context: never the headline's failure
            extra["entropy_routes_L24"] = {"error": repr(e)}
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
                "roofline": roof if roof is not None else extra["roofline_L24"], "cpu_baseline": cpu,
                "clocks": res["clocks"], "gpu_launches": res["launches_per_step"] * args.steps, **extra}
        if "e2e" in res:
            line["e2e"] = res["e2e"]
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
