"""Reduced density matrices of all pairs (all two-point Pauli correlators) and
the bond-entropy sweep through the C ABI against the oracle's RDM route."""
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


def pairs(L):
    return [(i, j) for i in range(1, L + 1) for j in range(i + 1, L + 1)]


@pytest.mark.parametrize("prec,atol", [("fp64", 1e-13), ("mixed", 2e-6)])
@pytest.mark.parametrize("L", [2, 7, 10])
def test_pair_rdms_match_oracle(prec, atol, L):
    psi = si.gaussian_state(L, 90 + L)
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec=prec)
    x = to_dev(psi, prec)
    ref = x.cpu().numpy().astype(np.complex128)
    r2, r1 = c.rdm_pairs(x)
    for p, (i, j) in enumerate(pairs(L)):
        np.testing.assert_allclose(r2[p], O.rdm_sites(ref, L, (i, j)), atol=atol)
    for i in range(1, L + 1):
        np.testing.assert_allclose(r1[i - 1], O.rdm_sites(ref, L, (i,)), atol=atol)


def test_pair_rdms_full_size_sampled():
    """L = 24, complex64: an entangled state from a short quench; three pairs against
    the oracle on the downloaded state, and every pair's trace, hermiticity and
    consistency with <sz_i sz_j>."""
    L = 24
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    x = c.new_state()
    c.init_basis_state(x, 0)
    c.krylov_evolve(x, 0.05, 4, 20)
    r2, r1 = c.rdm_pairs(x)
    ref = x.cpu().numpy().astype(np.complex128)
    ps = pairs(L)
    for (i, j) in ((1, 2), (3, 17), (23, 24)):
        np.testing.assert_allclose(r2[ps.index((i, j))], O.rdm_sites(ref, L, (i, j)), atol=2e-6)
    tr = np.einsum("pii->p", r2)
    np.testing.assert_allclose(tr, 1.0, atol=2e-5)
    np.testing.assert_allclose(r2, np.conj(np.transpose(r2, (0, 2, 1))), atol=0)
    zz = c.measure_corr(x)
    zzr = np.array([(r2[p][0, 0] - r2[p][1, 1] - r2[p][2, 2] + r2[p][3, 3]).real for p in range(len(ps))])
    np.testing.assert_allclose(zzr, [zz[i - 1, j - 1] for i, j in ps], atol=2e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L", [12, 17])
def test_entropy_sweep_matches_oracle(prec, L):
    psi = si.gaussian_state(L, 95)
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec=prec)
    x = to_dev(psi, prec)
    ref = x.cpu().numpy().astype(np.complex128)
    S = c.entropy_sweep(x)
    want = [O.entropy_from_spectrum(O.schmidt_spectrum_small(ref, L, l)) for l in range(1, L)]
    np.testing.assert_allclose(S, want, atol=1e-12 if prec == "fp64" else 1e-5)
