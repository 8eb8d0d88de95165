"""Krylov evolution on the three-pass H.psi layout (complex64 from L = 27: 64 KiB
tiles hold 13 bits, the first pass and two gathered passes cover 27) at a size
the oracle cannot evolve in test time.  The checks are what the mathematics
fixes at any size, on sampled rows, with the oracle's own pair-loop diagonal:
  * J = 0 from all up: every site rotates alone, amplitude of b =
    cos(ht)^(L-p) (-i sin(ht))^p with p = popcount(b); <sz_k> = cos 2ht,
    <sz_i sz_j> = cos^2 2ht (every flip bit of every pass);
  * h = 0: psi_b(t) = exp(-i E(b) t) psi_b(0) (the diagonal of every tile);
  * the full long-range quench against the FP64 form (whose three-pass layout
    starts at L = 24 and is checked against the oracle there)."""
import math

import numpy as np
import pytest
import torch

import seeded_inputs as si
from oracle import ed_oracle as O
from _gpu import TOL, seeded_device_state

pytestmark = pytest.mark.gpu

L = 27


def Chain(*a, **k):
    from paper_1802_10052_gb300 import Chain as _C
    return _C(*a, **k)


def sample_rows(rng, n_random=4000):
    low = [0] + [1 << k for k in range(L)] + [(1 << i) | (1 << j) for i in range(L) for j in range(i + 1, L)]
    return np.unique(np.concatenate([np.array(low, dtype=np.int64), rng.integers(0, 1 << L, size=n_random)]))


def fetch(x, rows):
    idx = torch.from_numpy(rows).to(x.device)
    return x[idx].cpu().numpy().astype(np.complex128)


@pytest.mark.timeout(900)
def test_krylov_L27_zero_coupling_closed_form():
    h, dt, n, m = 0.8, 0.01, 10, 20
    c = Chain(L, couplings=[0.0] * (L - 1), h=h, prec="mixed")
    x = c.new_state()
    c.init_basis_state(x, 0)
    c.krylov_evolve(x, dt, n, m)
    t = n * dt
    sz, zz = c.measure_zz(x)
    np.testing.assert_allclose(sz, math.cos(2 * h * t), rtol=0, atol=TOL["mixed"])
    off = zz[~np.eye(L, dtype=bool)]
    np.testing.assert_allclose(off, math.cos(2 * h * t) ** 2, rtol=0, atol=TOL["mixed"])
    rows = sample_rows(np.random.default_rng(27))
    p = np.array([bin(int(b)).count("1") for b in rows])
    want = math.cos(h * t) ** (L - p) * (-1j * math.sin(h * t)) ** p
    got = fetch(x, rows)
    assert np.linalg.norm(got - want) <= TOL["mixed"] * np.linalg.norm(want)
    c.close()


@pytest.mark.timeout(900)
def test_krylov_L27_zero_field_phases():
    dt, n, m = 0.01, 5, 20
    Jr = O.coupling_table(L, 1.0, 1.5)
    c = Chain(L, J=1.0, alpha=1.5, h=0.0, prec="mixed")
    x = seeded_device_state(L, 2727, "mixed")
    rows = sample_rows(np.random.default_rng(28))
    x0 = fetch(x, rows)
    c.krylov_evolve(x, dt, n, m)
    want = np.exp(-1j * O.diagonal_energy(L, Jr, rows) * dt * n) * x0
    got = fetch(x, rows)
    assert np.linalg.norm(got - want) <= TOL["mixed"] * np.linalg.norm(want)
    c.close()


@pytest.mark.timeout(900)
def test_krylov_L27_lrqi_quench_mixed_against_fp64():
    dt, n, m = 0.01, 5, 20
    out = {}
    for prec in ("fp64", "mixed"):
        c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec=prec)
        x = c.new_state()
        c.init_basis_state(x, 0)
        c.krylov_evolve(x, dt, n, m)
        sz, zz = c.measure_zz(x)
        e, n2 = c.energy(x)
        out[prec] = (x.to(torch.complex128), sz, zz, e, n2)
        c.close()
        del x
        torch.cuda.empty_cache()
    xf, szf, zzf, ef, nf = out["fp64"]
    xm, szm, zzm, em, nm = out["mixed"]
    assert (torch.linalg.vector_norm(xm - xf) / torch.linalg.vector_norm(xf)).item() < TOL["mixed"]
    np.testing.assert_allclose(szm, szf, rtol=0, atol=TOL["mixed"])
    np.testing.assert_allclose(zzm, zzf, rtol=0, atol=TOL["mixed"])
    # the FP64 form conserves the norm and the all-up energy sum_r (L - r) J(r)
    e0 = sum((L - r) / r ** 1.5 for r in range(1, L))
    assert abs(nf - 1.0) < 1e-12 and abs(ef / nf - e0) < TOL["fp64"] * abs(e0)
    assert abs(em / nm - e0) < TOL["mixed"] * abs(e0)


@pytest.mark.timeout(900)
@pytest.mark.parametrize("Lc,prec,tol", [(26, "mixed", 1e-6), (24, "fp64", 1e-10)])
def test_lanczos_three_pass_nn_chain_jordan_wigner(Lc, prec, tol):
    """Ground energy of the open nearest-neighbour chain (J = 1, h = 2, gapped) on the
    three-pass layout (complex64 from L = 26, complex128 from L = 24) against the
    Jordan-Wigner closed form, which holds at any L."""
    c = Chain(Lc, couplings=[1.0] + [0.0] * (Lc - 2), h=2.0, prec=prec)
    c.set_reorth(0)
    x = seeded_device_state(Lc, 2600 + Lc, prec)
    E, res, it = c.lanczos_ground(x, tol=tol, max_iter=120, raise_on_noconv=(prec == "fp64"))
    want = O.jordan_wigner_ground_energy(Lc, 1.0, 2.0)
    assert abs(E - want) < TOL[prec] * abs(want), (E, want, res, it)
    c.close()
