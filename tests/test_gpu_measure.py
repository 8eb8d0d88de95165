"""Measurements through the C ABI against the oracle's reduced density matrices."""
import math

import numpy as np
import pytest
import torch

import seeded_inputs as si
from oracle import ed_oracle as O
from _gpu import TOL, rel, to_dev

pytestmark = pytest.mark.gpu


def Chain(*a, **k):
    from paper_1802_10052_gb300 import Chain as _C
    return _C(*a, **k)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L", [1, 2, 3, 5, 9, 10, 11, 14, 16])
def test_local_and_corr_match_rdm_route(L, prec):
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec=prec)
    psi = si.gaussian_state(L, 40 + L) * 0.9
    x = to_dev(psi, prec)
    ref_state = x.cpu().numpy().astype(np.complex128)
    tol = 1e-13 if prec == "fp64" else 1e-6
    want_sz, want_zz = O.measure_local(ref_state, L), O.measure_corr(ref_state, L)
    np.testing.assert_allclose(c.measure_local(x), want_sz, atol=tol)
    np.testing.assert_allclose(c.measure_corr(x), want_zz, atol=tol)
    sz, zz = c.measure_zz(x)
    np.testing.assert_allclose(sz, want_sz, atol=tol)
    np.testing.assert_allclose(zz, want_zz, atol=tol)


def test_measure_full_size_invariants():
    # L = 28: the all-up and Neel product states give exact +-1 patterns, and a
    # seeded random state satisfies <sz_i sz_i> = <psi|psi> with |<.>| <= norm
    from _gpu import seeded_device_state
    L = 28
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    x = c.new_state()
    c.init_basis_state(x, si.neel_index(L))
    sz, zz = c.measure_zz(x)
    np.testing.assert_allclose(sz, [(-1) ** k for k in range(L)], atol=0)
    np.testing.assert_allclose(zz, [[(-1) ** (i + j) for j in range(L)] for i in range(L)], atol=0)
    y = seeded_device_state(L, 3, "mixed")
    sz, zz = c.measure_zz(y)
    np.testing.assert_allclose(np.diag(zz), 1.0, atol=1e-6)
    assert np.all(np.abs(sz) < 1e-3) and np.all(np.abs(zz - np.diag(np.diag(zz))) < 1e-3)
    np.testing.assert_allclose(zz, zz.T, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_special_states(prec):
    L = 12
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec=prec)
    x = c.new_state()
    c.init_basis_state(x, si.neel_index(L))
    np.testing.assert_allclose(c.measure_local(x), [(-1) ** k for k in range(L)], atol=0)
    np.testing.assert_allclose(c.measure_corr(x), [[(-1) ** (i + j) for j in range(L)] for i in range(L)], atol=0)
    assert abs(c.schmidt_entropy(x)) < 1e-6
    g = to_dev(si.ghz_state(L), prec)
    np.testing.assert_allclose(c.measure_local(g), 0.0, atol=1e-7)
    np.testing.assert_allclose(c.measure_corr(g), 1.0, atol=1e-6)
    S, lam = c.schmidt_entropy(g, spectrum=True)
    assert abs(S - math.log(2.0)) < (1e-13 if prec == "fp64" else 1e-6)
    np.testing.assert_allclose(lam[:2], 0.5, atol=1e-7)
    np.testing.assert_allclose(lam[2:], 0.0, atol=1e-7)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,cut", [(2, 1), (3, -1), (3, 2), (8, -1), (9, -1), (9, 2), (9, 7), (12, -1), (13, -1), (13, 9),
                                   (16, 3), (16, 13), (18, 1), (18, 6), (17, 11)])
def test_schmidt_spectrum_matches_oracle(L, cut, prec):
    """Includes small blocks with long contractions (split over K on the CUDA cores)."""
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec=prec)
    psi = si.gaussian_state(L, 60 + L)
    x = to_dev(psi, prec)
    ref_state = x.cpu().numpy().astype(np.complex128)
    l = L // 2 if cut == -1 else cut
    want = O.schmidt_spectrum_small(ref_state, L, l)
    S, lam = c.schmidt_entropy(x, cut=cut, spectrum=True)
    n = 1 << min(l, L - l)
    tol = 1e-13 if prec == "fp64" else 1e-6
    np.testing.assert_allclose(lam, want[:n], atol=tol)
    assert abs(S - O.entropy_from_spectrum(want)) < (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_page_value_L20(prec):
    L = 20
    m = n = 1 << (L // 2)
    page = sum(1.0 / k for k in range(n + 1, m * n + 1)) - (m - 1) / (2.0 * n)
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec=prec)
    x = to_dev(si.gaussian_state(L, 7), prec)
    S, lam = c.schmidt_entropy(x, spectrum=True)
    assert abs(S - page) < 2e-3
    assert abs(lam.sum() - 1.0) < (1e-12 if prec == "fp64" else 1e-5)
    assert lam.min() > -1e-6


@pytest.mark.parametrize("L,cut", [(14, -1), (15, 7), (16, -1), (18, 8), (19, -1)])
def test_tensor_core_gram_matches_oracle(L, cut):
    """Half-chain spectrum with the Gram product on the tensor cores (tcgen05,
    3xTF32) against the oracle's eigvalsh(M M^dagger), and against the CUDA-core
    Gram product of the same state."""
    psi = si.gaussian_state(L, 80 + L)
    x = to_dev(psi, "mixed")
    ref_state = x.cpu().numpy().astype(np.complex128)
    l = L // 2 if cut == -1 else cut
    want = O.schmidt_spectrum_small(ref_state, L, l)
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec="mixed")
    c.set_entropy_method(0)  # eigenvalues of the Gram product itself
    c.set_gram_mode(2)
    S_tc, lam_tc = c.schmidt_entropy(x, cut=cut, spectrum=True)
    n = 1 << min(l, L - l)
    np.testing.assert_allclose(lam_tc, want[:n], atol=2e-6)
    assert abs(S_tc - O.entropy_from_spectrum(want)) < 1e-5
    c.set_gram_mode(1)
    S_cc, lam_cc = c.schmidt_entropy(x, cut=cut, spectrum=True)
    np.testing.assert_allclose(lam_tc, lam_cc, atol=2e-6)


def test_tensor_core_gram_product_state_and_ghz():
    L = 16
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec="mixed")
    c.set_gram_mode(2)
    x = c.new_state()
    c.init_basis_state(x, si.neel_index(L))
    S, lam = c.schmidt_entropy(x, spectrum=True)
    assert abs(S) < 1e-6 and abs(lam[0] - 1.0) < 1e-6
    g = to_dev(si.ghz_state(L), "mixed")
    S, lam = c.schmidt_entropy(g, spectrum=True)
    assert abs(S - math.log(2.0)) < 1e-6
    np.testing.assert_allclose(lam[:2], 0.5, atol=1e-7)


def test_mixed_spectrum_of_nearly_rank_one_state_L24():
    """L = 24 quench state at t = 0.1 (FP64 evolution, rounded to complex64): rho
    is nearly rank one (4094 eigenvalues below 1e-7).  Gram route (method 0):
    the complex64 spectrum must be finite and sum to one (the library solver has
    returned non-finite values on such a matrix; then this library's reduction
    takes over).  Default route: S agrees with the FP64 form within the mixed
    tolerance."""
    L = 24
    c64 = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="fp64")
    x = c64.new_state()
    c64.init_basis_state(x, 0)
    c64.krylov_evolve(x, 0.01, 10, 20)
    S64 = c64.schmidt_entropy(x)
    y = x.to(torch.complex64)
    del x, c64
    torch.cuda.empty_cache()
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    c.set_entropy_method(0)
    _, lam = c.schmidt_entropy(y, spectrum=True)
    assert np.all(np.isfinite(lam))
    assert abs(lam.sum() - 1.0) < 1e-5
    assert abs(lam[0] - (1.0 - lam[1:].sum())) < 1e-5
    c.set_entropy_method(3)
    S, lam = c.schmidt_entropy(y, spectrum=True)
    assert np.all(np.isfinite(lam)) and abs(lam.sum() - 1.0) < 1e-6
    assert abs(S - S64) < TOL["mixed"]
