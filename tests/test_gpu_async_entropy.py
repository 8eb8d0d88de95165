"""Asynchronous bond entropy (Gram on the caller's stream, eigen-solve on the
handle's side stream) against the synchronous call and the oracle.  The
asynchronous call takes the Gram route (eigenvalues of rho), so the
synchronous results it is compared with take it too (entropy method 0)."""
import numpy as np
import pytest
import torch

import seeded_inputs as si
from oracle import ed_oracle as O
from _gpu import to_dev

pytestmark = pytest.mark.gpu


def Chain(*a, **k):
    from paper_1802_10052_gb300 import Chain as _C
    return _C(*a, **k)


def launches(c):
    import ctypes
    from paper_1802_10052_gb300 import _binding as B
    n = ctypes.c_int64()
    B.check(B.lib.osmps_ed_launch_count(c._h, ctypes.byref(n)), "osmps_ed_launch_count")
    return n.value


@pytest.mark.parametrize("prec,atol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_async_matches_sync_and_oracle(prec, atol):
    L = 12
    psi = si.gaussian_state(L, 7)
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec=prec)
    c.set_entropy_method(0)
    x = to_dev(psi, prec)
    S_sync, lam_sync = c.schmidt_entropy(x, cut=5, spectrum=True)
    p = c.schmidt_entropy_async(x, cut=5, spectrum=True)
    c.measure_wait()
    # same Gram kernel and eigen-solver on the same input: equal up to the solver's own run-to-run order
    assert abs(p.S - S_sync) <= 1e-12
    np.testing.assert_allclose(p.spectrum, lam_sync, rtol=0, atol=1e-12)
    ref = x.cpu().numpy().astype(np.complex128)
    lam_ref = O.schmidt_spectrum(ref, L, 5)
    assert abs(p.S - O.entropy_from_spectrum(lam_ref)) < atol
    np.testing.assert_allclose(p.spectrum, lam_ref, atol=atol)
    c.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_async_pipeline_with_state_overwritten(prec):
    """Three measurements along a Krylov evolution, each enqueued and the state
    evolved right after (the third call waits for the first slot); every
    result equals the synchronous entropy of the state it was enqueued on."""
    L = 16
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec=prec)
    c.set_entropy_method(0)
    x = c.new_state()
    c.init_basis_state(x, 0)
    snaps, pend = [], []
    for k in range(3):
        c.krylov_evolve(x, 0.1, 2, 16)
        snaps.append(x.clone())
        pend.append(c.schmidt_entropy_async(x))
        c.init_basis_state(x, 5)          # overwrite at once ...
        x.copy_(snaps[-1])                # ... and restore, both after the Gram in stream order
    with pytest.raises(RuntimeError):
        _ = pend[-1].S
    n0 = launches(c)
    c.measure_wait()
    for s, p in zip(snaps, pend):
        assert abs(p.S - c.schmidt_entropy(s)) <= 1e-12
    assert pend[-1].S > pend[0].S > 0.0
    assert launches(c) > n0          # the side stream's entropy kernels are added at the wait
    c.close()


def test_async_at_full_size_cut_half():
    """L = 24 complex64 (n = 4096 Schmidt values): async equals sync."""
    L = 24
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    c.set_entropy_method(0)
    x = c.new_state()
    c.init_basis_state(x, 0)
    c.krylov_evolve(x, 0.1, 3, 20)
    p = c.schmidt_entropy_async(x, spectrum=True)
    y = x.clone()
    c.krylov_evolve(x, 0.1, 1, 20)
    c.measure_wait()
    S, lam = c.schmidt_entropy(y, spectrum=True)
    assert abs(p.S - S) <= 1e-12
    np.testing.assert_allclose(p.spectrum, lam, rtol=0, atol=1e-12)
    assert abs(p.spectrum.sum() - 1.0) < 1e-4
    c.close()


def test_async_argument_errors():
    from paper_1802_10052_gb300 import OsmpsError
    c = Chain(8, J=1.0, alpha=None, h=1.0, prec="fp64")
    x = c.new_state()
    c.init_basis_state(x, 0)
    with pytest.raises(OsmpsError):
        c.schmidt_entropy_async(x, cut=8)
    c.measure_wait()          # nothing outstanding
    c.close()


# ---- this library's eigen-solver on a few CTAs (osmps_ed_set_async_eigensolver) ----

def own_entropy(c, x, cut=-1, ctas=16):
    c.set_async_eigensolver(ctas)
    p = c.schmidt_entropy_async(x, cut=cut, spectrum=True)
    c.measure_wait()
    return p.S, p.spectrum


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,cut", [(2, 1), (3, -1), (3, 2), (8, -1), (9, 2), (9, 7), (12, -1), (13, -1), (13, 9)])
def test_own_solver_matches_oracle(L, cut, prec):
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec=prec)
    x = to_dev(si.gaussian_state(L, 60 + L), prec)
    ref = x.cpu().numpy().astype(np.complex128)
    l = L // 2 if cut == -1 else cut
    want = O.schmidt_spectrum_small(ref, L, l)
    S, lam = own_entropy(c, x, cut)
    n = 1 << min(l, L - l)
    np.testing.assert_allclose(lam, want[:n], atol=1e-13 if prec == "fp64" else 1e-6)
    assert abs(S - O.entropy_from_spectrum(want)) < (1e-12 if prec == "fp64" else 1e-5)
    c.close()


@pytest.mark.parametrize("L,cut,ctas", [(14, -1, 8), (16, -1, 16), (19, -1, 24), (18, 8, 152)])
def test_own_solver_tensor_core_gram_matches_oracle(L, cut, ctas):
    x = to_dev(si.gaussian_state(L, 80 + L), "mixed")
    ref = x.cpu().numpy().astype(np.complex128)
    l = L // 2 if cut == -1 else cut
    want = O.schmidt_spectrum_small(ref, L, l)
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec="mixed")
    S, lam = own_entropy(c, x, cut, ctas)
    n = 1 << min(l, L - l)
    np.testing.assert_allclose(lam, want[:n], atol=2e-6)
    assert abs(S - O.entropy_from_spectrum(want)) < 1e-5
    c.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_own_solver_page_value_and_special_states(prec):
    import math
    L = 20
    m = n = 1 << (L // 2)
    page = sum(1.0 / k for k in range(n + 1, m * n + 1)) - (m - 1) / (2.0 * n)
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec=prec)
    x = to_dev(si.gaussian_state(L, 7), prec)
    S, lam = own_entropy(c, x)
    assert abs(S - page) < 2e-3
    assert abs(lam.sum() - 1.0) < (1e-12 if prec == "fp64" else 1e-5)
    c.init_basis_state(x, si.neel_index(L))
    S, lam = own_entropy(c, x)
    assert abs(S) < 1e-6 and abs(lam[0] - 1.0) < 1e-6
    g = to_dev(si.ghz_state(L), prec)
    S, lam = own_entropy(c, g)
    assert abs(S - math.log(2.0)) < (1e-12 if prec == "fp64" else 1e-6)
    np.testing.assert_allclose(lam[:2], 0.5, atol=1e-7)
    np.testing.assert_allclose(lam[2:], 0.0, atol=1e-7)
    c.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_own_solver_pipeline_against_library(prec, tol):
    """Three overlapped measurements along an evolution on the own solver (two
    slots, the third call waits for the first), each against the library
    solver's synchronous entropy of the same stored state."""
    L = 16
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec=prec)
    c.set_entropy_method(0)
    c.set_async_eigensolver(16)
    x = c.new_state()
    c.init_basis_state(x, 0)
    snaps, pend = [], []
    for _ in range(3):
        c.krylov_evolve(x, 0.1, 2, 16)
        snaps.append(x.clone())
        pend.append(c.schmidt_entropy_async(x, spectrum=True))
    c.measure_wait()
    for s, p in zip(snaps, pend):
        S, lam = c.schmidt_entropy(s, spectrum=True)
        assert abs(p.S - S) < tol
        np.testing.assert_allclose(p.spectrum, lam, atol=tol)
    c.set_async_eigensolver(0)
    p = c.schmidt_entropy_async(snaps[-1])
    c.measure_wait()
    assert abs(p.S - pend[-1].S) < tol
    c.close()


def test_own_solver_full_size_quench():
    """L = 24 complex64 quench state (n = 4096): own solver on 16 CTAs against the
    library solver on the same Gram product: the Schmidt values above 1e-4 to
    2e-6 and the trace.  Both are FP32 eigen-solvers of the FP32 Gram product,
    whose thousands of eigenvalues below 1e-7 are noise at that level; S of
    such a state is taken from the default (Rayleigh) route instead, which is
    checked against the FP64 form in test_gpu_entropy_rayleigh.py."""
    L = 24
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    c.set_entropy_method(0)
    x = c.new_state()
    c.init_basis_state(x, 0)
    c.krylov_evolve(x, 0.1, 5, 20)
    S_lib, lam_lib = c.schmidt_entropy(x, spectrum=True)
    S, lam = own_entropy(c, x, -1, 16)
    big = lam_lib > 1e-4
    np.testing.assert_allclose(lam[big], lam_lib[big], atol=2e-6)
    assert abs(lam.sum() - 1.0) < 1e-5
    c.close()
