"""Schmidt values as Rayleigh quotients of the Gram product's eigenvectors
(osmps_ed_set_entropy_method(2), the complex64 default where it applies)
against the oracle's spectrum (Sec. IV, bond entropy), and the accuracy it
keeps for weakly entangled complex64 states."""
import math

import numpy as np
import pytest
import torch

import seeded_inputs as si
from oracle import ed_oracle as O
from _gpu import TOL, to_dev

pytestmark = pytest.mark.gpu


def Chain(*a, **k):
    from paper_1802_10052_gb300 import Chain as _C
    return _C(*a, **k)


@pytest.mark.parametrize("L,cut", [(14, -1), (16, 8), (17, 8), (17, 9), (18, 7), (18, 11), (20, 10)])
def test_rayleigh_matches_oracle(L, cut):
    """Both orientations (left block the smaller: rows of M; the larger: columns),
    blocks of 128..1024 rows; the explicit method equals the automatic choice."""
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec="mixed")
    x = to_dev(si.gaussian_state(L, 90 + L), "mixed")
    ref = x.cpu().numpy().astype(np.complex128)
    l = L // 2 if cut == -1 else cut
    want = O.schmidt_spectrum_small(ref, L, l)
    S, lam = c.schmidt_entropy(x, cut=cut, spectrum=True)
    assert len(lam) == 1 << min(l, L - l)
    assert np.all(np.diff(lam) <= 0.0)
    np.testing.assert_allclose(lam, want, rtol=0, atol=1e-7)
    assert abs(S - O.entropy_from_spectrum(want)) < TOL["mixed"]
    c.set_entropy_method(2)
    S2, lam2 = c.schmidt_entropy(x, cut=cut, spectrum=True)
    assert S2 == S
    np.testing.assert_array_equal(lam2, lam)
    c.close()


@pytest.mark.parametrize("steps", [10, 50, 200])
def test_rayleigh_complex64_quench_L24_accuracy(steps):
    """The L = 24 quench (alpha = 1.5, h = 0.8, all up) at t = 0.1, 0.5, 2 evolved in
    FP64 and rounded to complex64: the default complex64 entropy meets the FP64
    entropy within the mixed tolerance (rounding the state alone moves S by
    ~1e-8; eigenvalues of the FP32 Gram product are off by up to ~2e-5 here)."""
    L = 24
    c64 = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="fp64")
    x = c64.new_state()
    c64.init_basis_state(x, 0)
    c64.krylov_evolve(x, 0.01, steps, 20)
    S64, lam64 = c64.schmidt_entropy(x, spectrum=True)
    y = x.to(torch.complex64)
    del x, c64
    torch.cuda.empty_cache()
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    S, lam = c.schmidt_entropy(y, spectrum=True)
    assert np.all(np.isfinite(lam)) and np.all(lam >= 0.0) and np.all(np.diff(lam) <= 0.0)
    assert abs(lam.sum() - 1.0) < 1e-6
    assert abs(S - S64) < TOL["mixed"]
    # values closer together than the FP32 eigenvectors resolve (~1e-7) come out
    # averaged within their cluster; the spectrum stays within the mixed tolerance
    np.testing.assert_allclose(lam[:64], lam64[:64], rtol=0, atol=1e-6)
    c.close()


def test_rayleigh_product_and_ghz_states():
    L = 16
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    x = c.new_state()
    c.init_basis_state(x, si.neel_index(L))
    S, lam = c.schmidt_entropy(x, spectrum=True)
    assert abs(S) < 1e-6 and abs(lam[0] - 1.0) < 1e-7 and np.all(np.abs(lam[1:]) < 1e-7)
    g = to_dev(si.ghz_state(L), "mixed")
    S, lam = c.schmidt_entropy(g, spectrum=True)
    assert abs(S - math.log(2.0)) < TOL["mixed"]
    np.testing.assert_allclose(lam[:2], 0.5, atol=1e-7)
    np.testing.assert_allclose(lam[2:], 0.0, atol=1e-7)
    c.close()


def test_rayleigh_not_for_fp64_or_small_blocks():
    from paper_1802_10052_gb300 import OsmpsError
    c = Chain(12, J=1.0, alpha=1.5, h=0.8, prec="fp64")
    c.set_entropy_method(2)
    x = to_dev(si.gaussian_state(12, 3), "fp64")
    with pytest.raises(OsmpsError):
        c.schmidt_entropy(x)
    c.close()
    c = Chain(12, J=1.0, alpha=1.5, h=0.8, prec="mixed")  # 64 x 64 blocks: below one tensor-core tile
    c.set_entropy_method(2)
    x = to_dev(si.gaussian_state(12, 3), "mixed")
    with pytest.raises(OsmpsError):
        c.schmidt_entropy(x)
    c.set_entropy_method(3)
    ref = x.cpu().numpy().astype(np.complex128)
    assert abs(c.schmidt_entropy(x) - O.schmidt_entropy(ref, 12)) < TOL["mixed"]
    c.close()


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-8, 1e-19, 1e-21])
def test_rayleigh_nearly_product_states(eps):
    """All-up plus eps times a Gaussian state (L = 16): the Gram product's entries
    run down into FP32 subnormals.  The default route gives a finite spectrum and
    S within the mixed tolerance of the oracle's S of the same complex64 state
    (falling back to the singular values where the library's eigenvectors are not
    finite)."""
    L = 16
    psi = si.basis_state(L, 0) + eps * si.gaussian_state(L, 16)
    psi = psi / np.linalg.norm(psi)
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    x = to_dev(psi, "mixed")
    ref = x.cpu().numpy().astype(np.complex128)
    S, lam = c.schmidt_entropy(x, spectrum=True)
    assert np.all(np.isfinite(lam)) and math.isfinite(S)
    assert abs(S - O.schmidt_entropy(ref, L)) < TOL["mixed"]
    c.close()


@pytest.mark.parametrize("threads", [256, 512])
def test_rayleigh_on_quench_states_of_both_pass_shapes(threads):
    """The L = 16 quench (alpha = 1.5, h = 0.8, all-up, m = 20, dt = 0.01) after 10,
    20 and 30 steps with either H.psi CTA shape; the two shapes round differently,
    and one of the resulting states made the library return non-finite
    eigenvectors.  S against the oracle's S of the state the GPU holds."""
    L = 16
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    c.set_pass_threads(threads)
    x = c.new_state()
    c.init_basis_state(x, 0)
    for _ in range(3):
        c.krylov_evolve(x, 0.01, 10, 20)
        ref = x.cpu().numpy().astype(np.complex128)
        S, lam = c.schmidt_entropy(x, spectrum=True)
        assert np.all(np.isfinite(lam))
        assert abs(S - O.schmidt_entropy(ref, L)) < TOL["mixed"]
    c.close()
