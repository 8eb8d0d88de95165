"""Schmidt values on the dominant subspace (osmps_ed_set_entropy_method(4), the
complex64 default for blocks of 512..8192 rows) against the oracle's spectrum
(Sec. IV, bond entropy): weakly entangled quench states, both block
orientations, the fallback to the full route for strongly entangled states, and
the accuracy against the FP64 form at the L = 24 quench."""
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


def quench_state(L, steps, prec="mixed"):
    """The long-range quench (alpha = 1.5, h = 0.8) from all up after steps of dt = 0.01."""
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec=prec)
    x = c.new_state()
    c.init_basis_state(x, 0)
    c.krylov_evolve(x, 0.01, steps, 20)
    return c, x


@pytest.mark.parametrize("L,cut", [(18, 9), (20, 10), (20, 9), (22, 13), (21, 10), (21, 11)])
def test_subspace_matches_oracle_on_quench_states(L, cut):
    """Both orientations (n = 512..1024 rows): S within the mixed tolerance of the
    oracle's S of the same complex64 state, the leading values within 1e-7, the
    values summing to the norm, and method 4 equal to the automatic choice."""
    c, x = quench_state(L, 150)
    ref = x.cpu().numpy().astype(np.complex128)
    want = O.schmidt_spectrum_small(ref, L, cut)
    S, lam = c.schmidt_entropy(x, cut=cut, spectrum=True)
    assert len(lam) == 1 << min(cut, L - cut)
    assert np.all(np.isfinite(lam)) and np.all(lam >= 0.0) and np.all(np.diff(lam) <= 0.0)
    assert abs(S - O.entropy_from_spectrum(want)) < TOL["mixed"]
    np.testing.assert_allclose(lam[:32], want[:32], rtol=0, atol=1e-7)
    assert abs(lam.sum() - np.sum(want)) < 1e-6
    c2 = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    c2.set_entropy_method(4)
    S4, lam4 = c2.schmidt_entropy(x, cut=cut, spectrum=True)
    assert S4 == S
    np.testing.assert_array_equal(lam4, lam)
    c.close()
    c2.close()


@pytest.mark.parametrize("L,cut", [(18, 9), (20, 10), (22, 13)])
def test_subspace_falls_back_for_entangled_states(L, cut):
    """A Gaussian state (nearly maximal entanglement): no affordable subspace holds
    its weight, and the call returns the full route's values."""
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec="mixed")
    x = to_dev(si.gaussian_state(L, 70 + L), "mixed")
    ref = x.cpu().numpy().astype(np.complex128)
    want = O.schmidt_spectrum_small(ref, L, cut)
    c.set_entropy_method(4)
    S, lam = c.schmidt_entropy(x, cut=cut, spectrum=True)
    np.testing.assert_allclose(lam, want, rtol=0, atol=1e-7)
    assert abs(S - O.entropy_from_spectrum(want)) < TOL["mixed"]
    c.set_entropy_method(2)
    S2, lam2 = c.schmidt_entropy(x, cut=cut, spectrum=True)
    assert S2 == S
    c.close()


def test_subspace_product_and_ghz_states():
    """L = 20: a product state (one value 1) and the GHZ state (two values 1/2)."""
    L = 20
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    c.set_entropy_method(4)
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


@pytest.mark.parametrize("steps", [10, 100, 250, 500])
def test_subspace_quench_L24_against_fp64(steps):
    """The L = 24 quench at t = 0.1, 1, 2.5, 5 evolved in FP64 and rounded to
    complex64: the default complex64 entropy (dominant subspace) within the mixed
    tolerance of the FP64 entropy, its leading values within 1e-6, and the values
    summing to the norm within 1e-6."""
    L = 24
    c64, x = quench_state(L, steps, "fp64")
    S64, lam64 = c64.schmidt_entropy(x, spectrum=True)
    y = x.to(torch.complex64)
    del x
    c64.close()
    torch.cuda.empty_cache()
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    S, lam = c.schmidt_entropy(y, spectrum=True)
    assert np.all(np.isfinite(lam)) and np.all(lam >= 0.0) and np.all(np.diff(lam) <= 0.0)
    assert abs(lam.sum() - 1.0) < 1e-6
    assert abs(S - S64) < TOL["mixed"]
    np.testing.assert_allclose(lam[:64], lam64[:64], rtol=0, atol=1e-6)
    # a second call starts from the dimension the first one found
    S2 = c.schmidt_entropy(y)
    assert abs(S2 - S64) < TOL["mixed"]
    c.close()


def test_subspace_not_for_small_blocks():
    from paper_1802_10052_gb300 import OsmpsError
    for prec in ("mixed", "fp64"):
        c = Chain(16, J=1.0, alpha=1.5, h=0.8, prec=prec)  # 256 x 256 blocks: below the route's range
        c.set_entropy_method(4)
        x = to_dev(si.gaussian_state(16, 3), prec)
        with pytest.raises(OsmpsError):
            c.schmidt_entropy(x)
        c.close()


@pytest.mark.parametrize("L,cut", [(18, 9), (20, 10), (22, 13)])
def test_subspace_fp64_matches_oracle(L, cut):
    """complex128 quench states (the residual bound is 2e-12 of the trace there): S
    within the FP64 tolerance of the oracle's S, the leading values within 1e-12."""
    c, x = quench_state(L, 150, "fp64")
    ref = x.cpu().numpy()
    want = O.schmidt_spectrum_small(ref, L, cut)
    S, lam = c.schmidt_entropy(x, cut=cut, spectrum=True)
    assert abs(S - O.entropy_from_spectrum(want)) < TOL["fp64"]
    np.testing.assert_allclose(lam[:32], want[:32], rtol=0, atol=1e-12)
    # the values hold all but the uncaptured weight, at most 2e-12 of the trace
    assert abs(lam.sum() - np.sum(want)) < 2e-12 + 1e-14
    # a second call starts from the dimension the first one found (a different
    # subspace; the uncaptured share of S, w (1 + ln(n / w)) <= 7e-11 for w = 2e-12,
    # may differ between the two): within the FP64 tolerance of the oracle too
    c.set_entropy_method(4)
    S4 = c.schmidt_entropy(x, cut=cut)
    assert abs(S4 - O.entropy_from_spectrum(want)) < TOL["fp64"]
    c.close()


def test_subspace_fp64_falls_back_to_the_gram_route():
    """A complex128 Gaussian state: the FP64 Gram eigenvalues."""
    L = 18
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec="fp64")
    x = to_dev(si.gaussian_state(L, 41), "fp64")
    want = O.schmidt_spectrum_small(x.cpu().numpy(), L, 9)
    S, lam = c.schmidt_entropy(x, spectrum=True)
    np.testing.assert_allclose(lam, want, rtol=0, atol=1e-13)
    assert abs(S - O.entropy_from_spectrum(want)) < TOL["fp64"]
    c.set_entropy_method(0)
    assert c.schmidt_entropy(x) == S
    c.close()
