"""Schmidt values as squared singular values of the block matrix M
(osmps_ed_set_entropy_method(1)) against the oracle, and the accuracy it
buys for weakly entangled complex64 states."""
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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,cut", [(2, 1), (9, 2), (9, 7), (12, -1), (13, 9), (20, 17), (20, 3)])
def test_svd_method_matches_oracle(L, cut, prec):
    """Both orientations of M (left block smaller: copied as is; larger: transposed)."""
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec=prec)
    c.set_entropy_method(1)
    x = to_dev(si.gaussian_state(L, 70 + L), prec)
    ref = x.cpu().numpy().astype(np.complex128)
    l = L // 2 if cut == -1 else cut
    want = O.schmidt_spectrum_small(ref, L, l)
    S, lam = c.schmidt_entropy(x, cut=cut, spectrum=True)
    assert len(lam) == 1 << min(l, L - l)
    np.testing.assert_allclose(lam, want, atol=1e-13 if prec == "fp64" else 1e-6)
    assert abs(S - O.entropy_from_spectrum(want)) < (1e-12 if prec == "fp64" else 1e-6)
    c.close()


def test_svd_method_complex64_quench_L24_accuracy():
    """L = 24 quench state at t = 0.5 (FP64 evolution, rounded to complex64):
    the singular-value route meets the FP64 entropy to 1e-6 (measured 1.3e-7;
    rounding the state alone moves S by ~1e-8; the Gram route is off by
    ~2e-5 here)."""
    L = 24
    c64 = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="fp64")
    x = c64.new_state()
    c64.init_basis_state(x, 0)
    c64.krylov_evolve(x, 0.01, 50, 20)
    S64 = c64.schmidt_entropy(x)
    y = x.to(torch.complex64)
    del x, c64
    torch.cuda.empty_cache()
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    c.set_entropy_method(1)
    S, lam = c.schmidt_entropy(y, spectrum=True)
    assert np.all(np.isfinite(lam)) and np.all(lam >= 0.0) and np.all(np.diff(lam) <= 0.0)
    assert abs(lam.sum() - 1.0) < 1e-5
    assert abs(S - S64) < 1e-6
    from paper_1802_10052_gb300 import OsmpsError
    with pytest.raises(OsmpsError):
        c.schmidt_entropy_async(y)
    c.close()
