"""Trotter evolution (Sec. III.C) and layers of two-site gates (App. C) through
the C ABI against the oracle's tensordot application of the same two-site
propagators, plus closed forms and invariants at full size."""
import math

import numpy as np
import pytest

import seeded_inputs as si
from oracle import ed_oracle as O
from _gpu import TOL, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


def Chain(*a, **k):
    from paper_1802_10052_gb300 import Chain as _C
    return _C(*a, **k)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,order", [(8, 1), (8, 2), (8, 4), (11, 2), (11, 4), (16, 4)])
def test_trotter_matches_oracle(prec, L, order):
    rng = np.random.Generator(np.random.Philox(60 + L))
    hs = rng.uniform(-1.2, 1.2, size=L)  # site fields, signed
    J1 = -0.9
    psi = si.gaussian_state(L, 61 + L)
    want = O.trotter_evolve_tensor(psi, L, J1, hs, 0.07, 4, order)
    c = Chain(L, couplings=[J1] + [0.0] * (L - 2), prec=prec)
    c.set_site_fields(hs)
    x = to_dev(psi, prec)
    c.trotter_evolve(x, 0.07, 4, order)
    assert rel(to_host(x), want) < TOL[prec]


def haar_unitaries(rng, k):
    """k Haar-random 4 x 4 unitaries (QR of complex Gaussians, phases fixed)."""
    out = []
    for _ in range(k):
        z = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
        q, r = np.linalg.qr(z)
        out.append(q * (np.diag(r) / np.abs(np.diag(r))))
    return np.array(out)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L", [9, 14])
def test_gate_layer_matches_oracle(prec, L):
    """Unitary gates (the circuits of App. C) within the stated tolerance."""
    rng = np.random.Generator(np.random.Philox(70 + L))
    psi = si.gaussian_state(L, 71 + L)
    sites = [1, 3, 6, L - 1] if L > 9 else [1, 4, 6, 8]
    U = haar_unitaries(rng, len(sites))
    want = psi
    for s, u in zip(sites, U):
        want = O.apply_two_site(want, L, s, u)
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec=prec)
    x = to_dev(psi, prec)
    c.apply_gates(x, sites, U)
    assert rel(to_host(x), want) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_general_gate_layer_within_rounding_bound(prec):
    """Non-unitary gates (complex Gaussian entries): every output amplitude is a
    four-term complex sum per gate, so the computed layer obeys the a-priori
    bound |y_hat - y| <= ((1 + g)^(m+1) - 1) |U_m|...|U_1| |psi| elementwise
    (g = 10 u bounds one gate's 8-term real dot products, u the unit roundoff;
    the extra factor covers rounding psi to the state type; Higham, Accuracy
    and Stability of Numerical Algorithms, Sec. 3.5)."""
    L = 12
    rng = np.random.Generator(np.random.Philox(77))
    psi = si.gaussian_state(L, 78)
    sites = [1, 4, 6, 11]
    U = rng.standard_normal((4, 4, 4)) + 1j * rng.standard_normal((4, 4, 4))
    want, bound = psi, np.abs(psi)
    for s, u in zip(sites, U):
        want = O.apply_two_site(want, L, s, u)
        bound = np.abs(O.apply_two_site(bound, L, s, np.abs(u)))
    c = Chain(L, J=1.0, alpha=1.0, h=1.0, prec=prec)
    x = to_dev(psi, prec)
    c.apply_gates(x, sites, U)
    u_ro = 2.0 ** -24 if prec == "mixed" else 2.0 ** -53
    g = 10 * u_ro
    err = np.abs(to_host(x) - want)
    assert np.all(err <= ((1 + g) ** (len(sites) + 1) - 1) * bound + 1e-300)


def test_gate_layer_rejects_overlapping_bonds_and_long_range_trotter():
    from paper_1802_10052_gb300 import OsmpsError
    c = Chain(8, J=1.0, alpha=1.5, h=1.0, prec="fp64")
    x = to_dev(si.basis_state(8, 0), "fp64")
    with pytest.raises(OsmpsError):
        c.apply_gates(x, [2, 3], np.stack([np.eye(4), np.eye(4)]))
    with pytest.raises(OsmpsError):  # long-range couplings: no bond decomposition
        c.trotter_evolve(x, 0.1, 1, 2)


def test_trotter_full_size_closed_form_and_norm():
    """L = 24, complex64: without bonds every layer term commutes, so from all up
    <sz_i(t)> = cos(2 h t) exactly; with bonds the gates are unitary (norm kept)."""
    L, h, dt, n = 24, 0.8, 0.05, 20
    c = Chain(L, couplings=[0.0] * (L - 1), h=h, prec="mixed")
    x = c.new_state()
    c.init_basis_state(x, 0)
    c.trotter_evolve(x, dt, n, 4)
    np.testing.assert_allclose(c.measure_local(x), math.cos(2 * h * dt * n), atol=2e-6)
    c2 = Chain(L, couplings=[1.0] + [0.0] * (L - 2), h=h, prec="mixed")
    y = c2.new_state()
    c2.init_basis_state(y, 0)
    c2.trotter_evolve(y, dt, n, 2)
    e0, n0 = c2.energy(y)
    # complex64: each window pass rounds the rotated amplitudes (~6e-8 relative); 20 steps x
    # 2 layers x 6 windows = 240 passes
    assert abs(n0 - 1.0) < 240 * 2e-7
