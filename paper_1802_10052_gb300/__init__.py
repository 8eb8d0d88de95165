"""GB300-native exact diagonalization of spin-1/2 chains (arXiv:1802.10052 hot path).

Python front end of libosmps_ed: the same calls as the C ABI in
include/osmps_ed.h, taking torch CUDA tensors (complex128 for ``prec="fp64"``,
complex64 for ``prec="mixed"``) as state buffers.  PyTorch only provides device
memory and the CUDA stream; all computation runs in the library's kernels.

    chain = Chain(L=24, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    psi = chain.new_state()
    chain.init_basis_state(psi, 0)            # all up
    err = chain.krylov_evolve(psi, dt=0.01, nsteps=10, m=20)
    sz = chain.measure_local(psi)
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from ._binding import (LIB_PATH, OSMPS_ENOCONV, OSMPS_FP64, OSMPS_MIXED, OSMPS_OK, OsmpsError, check, lib)

__all__ = ["Chain", "ChainBatch", "FinalEnergy", "PendingEntropy", "OsmpsError", "LIB_PATH", "lib"]

_PREC = {"fp64": OSMPS_FP64, "mixed": OSMPS_MIXED}


def _torch():
    import torch

    return torch


def _dptr(t):
    return C.c_void_p(t.data_ptr())


class Chain:
    """One chain H = sum_{i<j} J(j-i) sz_i sz_j + sum_k h_k sx_k on the current CUDA device.

    ``couplings`` (length L-1, J(r) for r = 1..L-1) overrides ``J``/``alpha``;
    ``alpha=None`` means nearest neighbours only.  Signs are taken as given.
    """

    def __init__(self, L, J=1.0, alpha=None, h=1.0, couplings=None, prec="fp64", stream=None):
        torch = _torch()
        self.L = int(L)
        self.prec = prec
        self.dtype = torch.complex128 if prec == "fp64" else torch.complex64
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        if couplings is not None:
            arr = (C.c_double * max(self.L - 1, 1))(*[float(x) for x in couplings])
            cp = C.cast(arr, C.POINTER(C.c_double))
        else:
            cp = None
        a = -1.0 if alpha is None else float(alpha)
        handle = C.c_void_p()
        check(lib.osmps_ed_create(self.L, cp, float(J), a, float(h), _PREC[prec],
                                  C.c_void_p(self._stream.cuda_stream), C.byref(handle)), "osmps_ed_create")
        self._h = handle

    # ---- lifetime -------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib.osmps_ed_measure_wait(self._h)
            lib.osmps_ed_destroy(self._h)
            self._h = None
            self._pending = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- configuration --------------------------------------------------
    @property
    def D(self):
        return 1 << self.L

    def set_stream(self, stream):
        self._stream = stream
        check(lib.osmps_ed_set_stream(self._h, C.c_void_p(stream.cuda_stream)), "osmps_ed_set_stream")

    def set_field(self, h):
        check(lib.osmps_ed_set_field(self._h, float(h)), "osmps_ed_set_field")

    def set_site_fields(self, h_sites):
        arr = (C.c_double * self.L)(*[float(x) for x in h_sites])
        check(lib.osmps_ed_set_site_fields(self._h, arr), "osmps_ed_set_site_fields")

    def set_reorth(self, mode):
        check(lib.osmps_ed_set_reorth(self._h, int(mode)), "osmps_ed_set_reorth")

    def set_gram_mode(self, mode):
        """0 automatic, 1 CUDA cores, 2 tensor cores (tcgen05, 3xTF32; complex64 only)."""
        check(lib.osmps_ed_set_gram_mode(self._h, int(mode)), "osmps_ed_set_gram_mode")

    def timing_enable(self, on=True):
        check(lib.osmps_ed_timing_enable(self._h, 1 if on else 0), "osmps_ed_timing_enable")

    def timing_read(self, reset=True):
        """(total ms, number of H.psi products) recorded since the last reset."""
        ms, n = C.c_double(), C.c_int64()
        check(lib.osmps_ed_timing_read(self._h, C.byref(ms), C.byref(n), 1 if reset else 0), "osmps_ed_timing_read")
        return ms.value, n.value

    def device_bytes(self):
        v = C.c_uint64()
        check(lib.osmps_ed_device_bytes(self._h, C.byref(v)), "osmps_ed_device_bytes")
        return v.value

    # ---- states ---------------------------------------------------------
    def new_state(self):
        torch = _torch()
        return torch.empty(self.D, dtype=self.dtype, device="cuda")

    def _check_state(self, t):
        if t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous() or t.numel() != self.D:
            raise ValueError(f"state must be a contiguous CUDA {self.dtype} tensor of {self.D} elements")

    def init_basis_state(self, psi, b):
        self._check_state(psi)
        check(lib.osmps_ed_init_basis_state(self._h, _dptr(psi), int(b)), "osmps_ed_init_basis_state")

    def upload(self, dst, src_host):
        self._check_state(dst)
        if src_host.dtype != self.dtype or src_host.numel() != self.D or not src_host.is_contiguous():
            raise ValueError("host buffer has the wrong type or size")
        check(lib.osmps_ed_upload(self._h, _dptr(dst), C.c_void_p(src_host.data_ptr())), "osmps_ed_upload")

    def download(self, dst_host, src):
        self._check_state(src)
        if dst_host.dtype != self.dtype or dst_host.numel() != self.D or not dst_host.is_contiguous():
            raise ValueError("host buffer has the wrong type or size")
        check(lib.osmps_ed_download(self._h, C.c_void_p(dst_host.data_ptr()), _dptr(src)), "osmps_ed_download")

    # ---- hot path -------------------------------------------------------
    def apply_H(self, psi, out):
        self._check_state(psi)
        self._check_state(out)
        check(lib.osmps_ed_apply_H(self._h, _dptr(psi), _dptr(out)), "osmps_ed_apply_H")

    def energy(self, psi):
        """Returns (<psi|H|psi>, <psi|psi>)."""
        self._check_state(psi)
        e, n = C.c_double(), C.c_double()
        check(lib.osmps_ed_energy(self._h, _dptr(psi), C.byref(e), C.byref(n)), "osmps_ed_energy")
        return e.value, n.value

    def lanczos_ground(self, psi, tol=1e-12, max_iter=300, raise_on_noconv=True):
        """In place: psi <- normalised ground state.  Returns (E, residual, iterations)."""
        self._check_state(psi)
        e, r, it = C.c_double(), C.c_double(), C.c_int()
        st = lib.osmps_ed_lanczos_ground(self._h, _dptr(psi), float(tol), int(max_iter), C.byref(e), C.byref(r),
                                         C.byref(it))
        allow = (OSMPS_OK,) if raise_on_noconv else (OSMPS_OK, OSMPS_ENOCONV)
        check(st, "osmps_ed_lanczos_ground", allow)
        return e.value, r.value, it.value

    def krylov_evolve(self, psi, dt, nsteps, m=20, tol=0.0):
        """In place: psi <- exp(-i H dt)^nsteps psi.  Returns the summed error estimate."""
        self._check_state(psi)
        err = C.c_double()
        check(lib.osmps_ed_krylov_evolve(self._h, _dptr(psi), float(dt), int(nsteps), int(m), float(tol),
                                         C.byref(err)), "osmps_ed_krylov_evolve")
        return err.value

    def adjoint_grad(self, psi0, h_steps, dt, m=20, h_target=1.0, stride=None, nquad=8, want_grad=True):
        """Loss <psi_N|H(h_target)|psi_N> after the steps exp(-i dt H(h_k)) from psi0, and
        (if want_grad) d loss/d h_k and d loss/d s (s = overall coupling scale).
        Returns (loss, grad_h ndarray, grad_scale) or (loss, None, None)."""
        self._check_state(psi0)
        hs = np.ascontiguousarray(np.asarray(h_steps, dtype=np.float64))
        n = hs.size
        stride = int(stride) if stride is not None else max(1, int(round(math.sqrt(n))))
        loss = C.c_double()
        gh = np.zeros(n, dtype=np.float64) if want_grad else None
        gs = C.c_double()
        hp = hs.ctypes.data_as(C.POINTER(C.c_double))
        gp = gh.ctypes.data_as(C.POINTER(C.c_double)) if want_grad else None
        check(lib.osmps_ed_adjoint_grad(self._h, _dptr(psi0), n, float(dt), hp, int(m), float(h_target), stride,
                                        int(nquad), C.byref(loss), gp, C.byref(gs) if want_grad else None),
              "osmps_ed_adjoint_grad")
        return (loss.value, gh, gs.value) if want_grad else (loss.value, None, None)

    def apply_gates(self, psi, sites, U):
        """In place: apply 4 x 4 gates U[i] (complex, basis 2 sigma_s + sigma_{s+1}) on the
        disjoint bonds (sites[i], sites[i] + 1)."""
        self._check_state(psi)
        sites = [int(x) for x in sites]
        n = len(sites)
        Ua = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).reshape(n, 4, 4)).view(np.float64).ravel()
        sa = (C.c_int * max(n, 1))(*sites)
        check(lib.osmps_ed_apply_gates(self._h, _dptr(psi), n, sa, Ua.ctypes.data_as(C.POINTER(C.c_double))),
              "osmps_ed_apply_gates")

    def trotter_evolve(self, psi, dt, nsteps, order=2):
        """In place: psi <- Trotter product (order 1, 2 or 4) of exp(-i H dt), nsteps times."""
        self._check_state(psi)
        check(lib.osmps_ed_trotter_evolve(self._h, _dptr(psi), float(dt), int(nsteps), int(order)),
              "osmps_ed_trotter_evolve")

    def rdm_pairs(self, psi):
        """(rho2, rho1): rho2[p] the 4 x 4 RDM of the p-th pair (1,2), (1,3), ..., (L-1,L)
        in the basis 2 sigma_i + sigma_j; rho1[i] the 2 x 2 RDM of site i+1."""
        self._check_state(psi)
        L = self.L
        npairs = L * (L - 1) // 2
        r2 = np.zeros(npairs * 32)
        r1 = np.zeros(L * 8)
        check(lib.osmps_ed_rdm_pairs(self._h, _dptr(psi), r2.ctypes.data_as(C.POINTER(C.c_double)),
                                     r1.ctypes.data_as(C.POINTER(C.c_double))), "osmps_ed_rdm_pairs")
        return r2.view(np.complex128).reshape(npairs, 4, 4), r1.view(np.complex128).reshape(L, 2, 2)

    def entropy_sweep(self, psi):
        """Bond entropy S(l) of every cut l = 1..L-1."""
        self._check_state(psi)
        S = np.zeros(self.L - 1)
        check(lib.osmps_ed_entropy_sweep(self._h, _dptr(psi), S.ctypes.data_as(C.POINTER(C.c_double))),
              "osmps_ed_entropy_sweep")
        return S

    def measure_local(self, psi):
        self._check_state(psi)
        out = np.zeros(self.L)
        check(lib.osmps_ed_measure_local(self._h, _dptr(psi), out.ctypes.data_as(C.POINTER(C.c_double))),
              "osmps_ed_measure_local")
        return out

    def measure_corr(self, psi):
        self._check_state(psi)
        out = np.zeros((self.L, self.L))
        check(lib.osmps_ed_measure_corr(self._h, _dptr(psi), out.ctypes.data_as(C.POINTER(C.c_double))),
              "osmps_ed_measure_corr")
        return out

    def measure_zz(self, psi):
        """(<sz_k> for k = 1..L, <sz_i sz_j> as L x L) from one pass."""
        self._check_state(psi)
        sz = np.zeros(self.L)
        zz = np.zeros((self.L, self.L))
        check(lib.osmps_ed_measure_zz(self._h, _dptr(psi), sz.ctypes.data_as(C.POINTER(C.c_double)),
                                      zz.ctypes.data_as(C.POINTER(C.c_double))), "osmps_ed_measure_zz")
        return sz, zz

    def schmidt_entropy(self, psi, cut=-1, spectrum=False):
        """Returns S, or (S, lambda descending) with spectrum=True."""
        self._check_state(psi)
        c = self.L // 2 if cut in (-1, None) else int(cut)
        n = 1 << min(c, self.L - c)
        lam = np.zeros(n) if spectrum else None
        S = C.c_double()
        lp = lam.ctypes.data_as(C.POINTER(C.c_double)) if spectrum else None
        check(lib.osmps_ed_schmidt_entropy(self._h, _dptr(psi), int(c), lp, C.byref(S)), "osmps_ed_schmidt_entropy")
        return (S.value, lam) if spectrum else S.value

    def set_sm_count(self, nsm=0):
        """Size the handle's grids for nsm SMs (0: all of the device)."""
        check(lib.osmps_ed_set_sm_count(self._h, int(nsm)), "osmps_ed_set_sm_count")

    def set_entropy_method(self, method):
        """0: eigenvalues of the Gram product; 1: singular values of M; 2: Rayleigh
        quotients of the Gram product's eigenvectors (complex64); 3: automatic (default);
        4: Rayleigh quotients on the dominant subspace (complex64, full route as fallback)."""
        check(lib.osmps_ed_set_entropy_method(self._h, int(method)), "osmps_ed_set_entropy_method")

    def set_flip_sums(self, mode):
        """complex128 flip sums: k >= 1 = exact 64-bit fixed-point sums in uniform-field passes
        flipping at least k bits (default 1), 0 = FP64 multiply-adds."""
        check(lib.osmps_ed_set_flip_sums(self._h, int(mode)), "osmps_ed_set_flip_sums")

    def set_lanczos_fold(self, on):
        """Krylov Lanczos steps in three launches (1, default) or five (0); bit-identical."""
        check(lib.osmps_ed_set_lanczos_fold(self._h, int(on)), "osmps_ed_set_lanczos_fold")

    def set_pass_threads(self, threads):
        """CTA shape of the H.psi passes: 256 (16 vectors per thread) or 512 (8)."""
        check(lib.osmps_ed_set_pass_threads(self._h, int(threads)), "osmps_ed_set_pass_threads")

    def set_prefetch(self, tiles):
        """L2 prefetch distance of the H.psi passes (tiles ahead; 0 = off)."""
        check(lib.osmps_ed_set_prefetch(self._h, int(tiles)), "osmps_ed_set_prefetch")

    def set_async_eigensolver(self, ctas=0):
        """Eigen-solver of schmidt_entropy_async: 0 = library routine on a worker
        thread, > 0 = this library's reduction on (at least) that many CTAs."""
        check(lib.osmps_ed_set_async_eigensolver(self._h, int(ctas)), "osmps_ed_set_async_eigensolver")

    def schmidt_entropy_async(self, psi, cut=-1, spectrum=False):
        """Enqueues the bond entropy of psi without blocking; psi may be changed
        right after.  Returns a PendingEntropy whose values are valid after
        measure_wait()."""
        self._check_state(psi)
        c = self.L // 2 if cut in (-1, None) else int(cut)
        n = 1 << min(c, self.L - c)
        p = PendingEntropy(n if spectrum else 0)
        lp = p._lam.ctypes.data_as(C.POINTER(C.c_double)) if spectrum else None
        check(lib.osmps_ed_schmidt_entropy_async(self._h, _dptr(psi), int(c), p._S.ctypes.data_as(
            C.POINTER(C.c_double)), lp), "osmps_ed_schmidt_entropy_async")
        if not hasattr(self, "_pending"):
            self._pending = []
        self._pending.append(p)
        return p

    def measure_wait(self):
        """Blocks until every pending asynchronous measurement has its values."""
        st = lib.osmps_ed_measure_wait(self._h)
        for p in getattr(self, "_pending", []):
            p._done = st == 0
        self._pending = []
        check(st, "osmps_ed_measure_wait")


class PendingEntropy:
    """Result of Chain.schmidt_entropy_async: S (and the Schmidt spectrum,
    descending, when asked for) once Chain.measure_wait() has returned."""

    def __init__(self, n):
        self._S = np.zeros(1)
        self._lam = np.zeros(n)
        self._done = False

    @property
    def S(self):
        if not self._done:
            raise RuntimeError("measurement pending: call Chain.measure_wait() first")
        return float(self._S[0])

    @property
    def spectrum(self):
        if not self._done:
            raise RuntimeError("measurement pending: call Chain.measure_wait() first")
        return self._lam


class ChainBatch:
    """Ground states of many independent chains in one persistent launch.

    Chain k: H_k = sum_{i<j} J[k]/|i-j|^alpha[k] sz_i sz_j + h[k] sum_i sx_i on L[k]
    sites (``alpha[k]`` None: nearest neighbours only).  States are packed in
    one tensor; chain k occupies ``psi[offsets[k]:offsets[k+1]]``.
    """

    def __init__(self, L, J, alpha, h, prec="mixed", max_iter=1000, stream=None):
        torch = _torch()
        n = len(L)
        self.n = n
        self.L = [int(x) for x in L]
        self.prec = prec
        self.dtype = torch.complex128 if prec == "fp64" else torch.complex64
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        Ja = (C.c_double * n)(*[float(x) for x in J])
        Aa = (C.c_double * n)(*[-1.0 if a is None else float(a) for a in alpha])
        Ha = (C.c_double * n)(*[float(x) for x in h])
        La = (C.c_int * n)(*self.L)
        handle = C.c_void_p()
        check(lib.osmps_ed_batch_create(n, La, Ja, Aa, Ha, _PREC[prec], int(max_iter),
                                        C.c_void_p(self._stream.cuda_stream), C.byref(handle)),
              "osmps_ed_batch_create")
        self._h = handle
        off = (C.c_uint64 * (n + 1))()
        check(lib.osmps_ed_batch_offsets(self._h, off), "osmps_ed_batch_offsets")
        self.offsets = np.array(off[:], dtype=np.int64)
        self.energy = torch.zeros(n, dtype=torch.float64, device="cuda")
        self.residual = torch.zeros(n, dtype=torch.float64, device="cuda")
        self.iters = torch.zeros(n, dtype=torch.int32, device="cuda")
        self.status = torch.zeros(n, dtype=torch.int32, device="cuda")

    def close(self):
        if getattr(self, "_h", None):
            lib.osmps_ed_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def total(self):
        return int(self.offsets[-1])

    def new_states(self):
        torch = _torch()
        return torch.empty(self.total, dtype=self.dtype, device="cuda")

    def view(self, psi, k):
        return psi[int(self.offsets[k]):int(self.offsets[k + 1])]

    def device_bytes(self):
        v = C.c_uint64()
        check(lib.osmps_ed_batch_device_bytes(self._h, C.byref(v)), "osmps_ed_batch_device_bytes")
        return v.value

    def set_graph(self, on=True):
        check(lib.osmps_ed_batch_set_graph(self._h, 1 if on else 0), "osmps_ed_batch_set_graph")

    def set_split(self, csize, lsplit=22):
        """Clusters of ``csize`` CTAs solve the chains with L >= ``lsplit`` (csize 1: none)."""
        check(lib.osmps_ed_batch_set_split(self._h, int(csize), int(lsplit)), "osmps_ed_batch_set_split")

    def get_split(self):
        cs, ls, gr = C.c_int(), C.c_int(), C.c_int()
        check(lib.osmps_ed_batch_get_split(self._h, C.byref(cs), C.byref(ls), C.byref(gr)), "osmps_ed_batch_get_split")
        return cs.value, ls.value, gr.value

    def autotune(self, psi, tol=1e-10):
        """Time the candidate work splits on these start vectors (psi is restored) and
        keep the fastest; returns (csize, lsplit, grid, best_ms)."""
        ms = C.c_double()
        check(lib.osmps_ed_batch_autotune(self._h, _dptr(psi), float(tol), C.byref(ms)), "osmps_ed_batch_autotune")
        return self.get_split() + (ms.value,)

    def launch_count(self):
        v = C.c_int64()
        check(lib.osmps_ed_batch_launch_count(self._h, C.byref(v)), "osmps_ed_batch_launch_count")
        return v.value

    def lanczos_ground_async(self, psi, tol=1e-10):
        """Enqueue the solve (start vectors in, ground states out); results land in
        the device tensors ``energy``, ``residual``, ``iters``, ``status``."""
        if psi.dtype != self.dtype or not psi.is_cuda or psi.numel() != self.total:
            raise ValueError("psi must be a packed CUDA state tensor of this batch")
        check(lib.osmps_ed_batch_lanczos_ground(self._h, _dptr(psi), float(tol), _dptr(self.energy),
                                                _dptr(self.residual), _dptr(self.iters), _dptr(self.status)),
              "osmps_ed_batch_lanczos_ground")

    def check(self):
        check(lib.osmps_ed_batch_check(self._h), "osmps_ed_batch_check")

    def lanczos_ground(self, psi, tol=1e-10):
        """Solve and return host arrays (energy, residual, iters, status)."""
        self.lanczos_ground_async(psi, tol)
        self.check()
        return (self.energy.cpu().numpy(), self.residual.cpu().numpy(), self.iters.cpu().numpy(),
                self.status.cpu().numpy())


def _make_final_energy():
    torch = _torch()

    class FinalEnergy(torch.autograd.Function):
        """loss = <psi_N|H(h_target)|psi_N> as a differentiable function of the per-step
        fields h (1-D float64 tensor) and the coupling scale s (0-D float64 tensor, the
        factor on the chain's couplings; pass ones to differentiate at the chain as built).
        The backward pass runs the adjoint sweep of the library (osmps_ed_adjoint_grad).
        Only s = 1 is supported (the chain's couplings are fixed at create)."""

        @staticmethod
        def forward(ctx, h, s, chain, psi0, dt, m, h_target):
            if float(s) != 1.0:
                raise ValueError("FinalEnergy differentiates at coupling scale 1 (build the chain with the couplings)")
            loss, _, _ = chain.adjoint_grad(psi0, h.detach().cpu().numpy(), dt, m, h_target, want_grad=False)
            ctx.chain, ctx.psi0, ctx.dt, ctx.m, ctx.h_target = chain, psi0, dt, m, h_target
            ctx.save_for_backward(h)
            return torch.tensor(loss, dtype=torch.float64)

        @staticmethod
        def backward(ctx, g):
            (h,) = ctx.saved_tensors
            _, gh, gs = ctx.chain.adjoint_grad(ctx.psi0, h.detach().cpu().numpy(), ctx.dt, ctx.m, ctx.h_target)
            gf = float(g)
            return (torch.from_numpy(gh * gf).to(h.dtype), torch.tensor(gs * gf, dtype=torch.float64),
                    None, None, None, None, None)

    return FinalEnergy


class _Lazy:
    def __init__(self):
        self._cls = None

    def apply(self, *a):
        if self._cls is None:
            self._cls = _make_final_energy()
        return self._cls.apply(*a)


FinalEnergy = _Lazy()
