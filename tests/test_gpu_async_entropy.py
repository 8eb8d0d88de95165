"""Asynchronous bond entropy (Gram on the caller's stream, eigen-solve on the
handle's side stream) against the synchronous call and the oracle."""
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


@pytest.mark.parametrize("prec,atol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_async_matches_sync_and_oracle(prec, atol):
    L = 12
    psi = si.gaussian_state(L, 7)
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec=prec)
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
