"""Lanczos ground state and Krylov evolution through the C ABI against the
FP64 oracle, closed forms and conservation laws."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import torch

import seeded_inputs as si
from oracle import ed_oracle as O
from _gpu import TOL, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


def Chain(*a, **k):
    from paper_1802_10052_gb300 import Chain as _C
    return _C(*a, **k)


# ---------------------------------------------------------------------------
# ground state
# ---------------------------------------------------------------------------

def test_nn_ground_L12_free_fermions():
    """Nearest-neighbour chain L=12, J=h=1 (Eq. HQI), seeded Gaussian start,
    residual 1e-12: energy against the Jordan-Wigner closed form."""
    w = si.WORKLOADS["nn_ground_L12"]
    c = Chain(w["L"], J=-1.0, alpha=None, h=-1.0, prec="fp64")
    x = to_dev(si.gaussian_state(w["L"], w["seed"]), "fp64")
    E, res, it = c.lanczos_ground(x, tol=w["tol"], max_iter=300)
    assert abs(E - (-14.925971109908655)) < 1e-12 * 15
    assert res <= w["tol"]
    # vector against the oracle's ground state (gap is large: unique up to phase)
    H = O.hamiltonian_csr(12, O.coupling_table(12, -1.0, None), -1.0)
    Eo, xo, _, _ = O.lanczos_ground(O.csr_matvec(H), si.gaussian_state(12, 1), tol=1e-12)
    xg = to_host(x)
    assert abs(abs(np.vdot(xo, xg)) - 1.0) < 1e-12
    assert abs(np.linalg.norm(xg) - 1.0) < 1e-13


def test_ground_mixed_precision_L12():
    c = Chain(12, J=-1.0, alpha=None, h=-1.0, prec="mixed")
    x = to_dev(si.gaussian_state(12, 1), "mixed")
    E, res, it = c.lanczos_ground(x, tol=1e-5, max_iter=300)
    assert abs(E - (-14.925971109908655)) < 1e-5 * 15
    assert res <= 1e-5


@pytest.mark.parametrize("L,alpha,h,J", [(8, 1.5, 0.8, 1.0), (10, 0.5, 0.3, -1.0), (9, 3.0, 1.7, 1.0)])
def test_ground_matches_dense_eigh(L, alpha, h, J):
    c = Chain(L, J=J, alpha=alpha, h=h, prec="fp64")
    e = np.linalg.eigvalsh(O.hamiltonian_dense(L, O.coupling_table(L, J, alpha), h))
    x = to_dev(si.gaussian_state(L, 3), "fp64")
    E, res, it = c.lanczos_ground(x, tol=1e-10, max_iter=400)
    assert E >= e[0] - 1e-10
    assert abs(E - e[0]) < 1e-10 * max(1.0, abs(e[0]))


def test_ground_pure_field_breakdown():
    # J = 0: E0 = -sum |h_k|; the Krylov space of a product-like start is small
    L = 11
    c = Chain(L, couplings=[0.0] * (L - 1), h=0.0, prec="fp64")
    hk = np.linspace(-1.0, 1.5, L)
    c.set_site_fields(hk)
    x = to_dev(si.gaussian_state(L, 5), "fp64")
    E, res, it = c.lanczos_ground(x, tol=1e-11, max_iter=200)
    assert abs(E + np.sum(np.abs(hk))) < 1e-11


# ---------------------------------------------------------------------------
# Krylov evolution
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_krylov_matches_oracle_steps(prec):
    L, alpha, h, m, dt = 13, 1.5, 0.8, 20, 0.01
    c = Chain(L, J=1.0, alpha=alpha, h=h, prec=prec)
    psi = si.gaussian_state(L, 17)
    x = to_dev(psi, prec)
    mv = O.RuleSetH(L, O.coupling_table(L, 1.0, alpha), h)
    ref = x.cpu().numpy().astype(np.complex128)
    for _ in range(10):
        ref, _ = O.krylov_step(mv, ref, dt, m)
    err = c.krylov_evolve(x, dt, 10, m)
    assert rel(to_host(x), ref) < (1e-11 if prec == "fp64" else 1e-5)
    assert err < 1e-8


@pytest.mark.parametrize("reorth", [0, 1])
def test_krylov_matches_dense_expm(reorth):
    L = 8
    Jr = O.coupling_table(L, 1.0, 1.5)
    Hd = O.hamiltonian_dense(L, Jr, 0.8)
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="fp64")
    c.set_reorth(reorth)
    psi = si.gaussian_state(L, 11)
    x = to_dev(psi, "fp64")
    c.krylov_evolve(x, 0.05, 10, 20)
    want = sla.expm(-1j * 0.5 * Hd) @ psi
    assert rel(to_host(x), want) < 1e-12


@pytest.mark.parametrize("prec,L", [("fp64", 20), ("mixed", 24)])
def test_pure_field_quench_closed_form(prec, L):
    """J = 0 from all-up: <sz_i(t)> = cos(2ht), <sz_i sz_j> = cos(2ht)^2, S = 0,
    at any L; m = L+3 > L+1 exercises the happy breakdown."""
    h, dt, n = 0.7, 0.05, 10
    c = Chain(L, couplings=[0.0] * (L - 1), h=h, prec=prec)
    x = c.new_state()
    c.init_basis_state(x, 0)
    c.krylov_evolve(x, dt, n, L + 3)
    t = dt * n
    cz = math.cos(2 * h * t)
    tol = 1e-12 if prec == "fp64" else 2e-6
    np.testing.assert_allclose(c.measure_local(x), cz, atol=tol)
    C = c.measure_corr(x)
    off = C[~np.eye(L, dtype=bool)]
    np.testing.assert_allclose(off, cz * cz, atol=tol)


def test_zero_field_phases():
    L = 10
    Jr = O.coupling_table(L, 1.0, 1.2)
    c = Chain(L, J=1.0, alpha=1.2, h=0.0, prec="fp64")
    psi = si.gaussian_state(L, 4)
    x = to_dev(psi, "fp64")
    c.krylov_evolve(x, 0.02, 20, 25)
    E = O.diagonal_energy(L, Jr, np.arange(1 << L))
    assert rel(to_host(x), np.exp(-1j * E * 0.4) * psi) < 1e-11


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_conservation_laws(prec):
    L = 18
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec=prec)
    x = to_dev(si.gaussian_state(L, 9), prec)
    e0, n0 = c.energy(x)
    flip = torch.arange(1 << L, device="cuda") ^ ((1 << L) - 1)
    p0 = torch.vdot(x, x[flip]).item()
    c.krylov_evolve(x, 0.02, 25, 20)
    e1, n1 = c.energy(x)
    p1 = torch.vdot(x, x[flip]).item()
    tol = 1e-10 if prec == "fp64" else 1e-5
    # scalars: |a - b| <= tol * max(|b|, 1)
    assert abs(n1 - n0) < tol * max(abs(n0), 1.0)
    assert abs(e1 - e0) < tol * max(abs(e0), 1.0)
    assert abs(p1 - p0) < tol * max(abs(p0), 1.0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lrqi_quench_short_horizon_vs_oracle(prec):
    """Long-range quench (alpha=1.5, h=0.8, all-up start, m=20, dt=0.01) at L=16,
    30 steps, with the measurements every 0.1 against the oracle."""
    L, alpha, h, m, dt = 16, 1.5, 0.8, 20, 0.01
    c = Chain(L, J=1.0, alpha=alpha, h=h, prec=prec)
    x = c.new_state()
    c.init_basis_state(x, 0)
    mv = O.RuleSetH(L, O.coupling_table(L, 1.0, alpha), h)
    ref = si.basis_state(L, 0)
    tol = TOL[prec]
    for block in range(3):
        for _ in range(10):
            ref, _ = O.krylov_step(mv, ref, dt, m)
        c.krylov_evolve(x, dt, 10, m)
        got = to_host(x)
        assert rel(got, ref) < tol
        np.testing.assert_allclose(c.measure_local(x), O.measure_local(ref, L), atol=tol)
        np.testing.assert_allclose(c.measure_corr(x), O.measure_corr(ref, L), atol=tol)
        S = c.schmidt_entropy(x)
        assert abs(S - O.schmidt_entropy(ref, L)) < tol * max(1.0, S)


def test_lrqi_quench_L24_two_steps_vs_oracle():
    """The L=24 long-range quench itself (alpha=1.5, h=0.8, m=20, dt=0.01): two
    steps from all-up in FP64 and mixed against the oracle's rule-set product."""
    L, alpha, h, m, dt = 24, 1.5, 0.8, 20, 0.01
    mv = O.RuleSetH(L, O.coupling_table(L, 1.0, alpha), h)
    ref = si.basis_state(L, 0)
    for _ in range(2):
        ref, _ = O.krylov_step(mv, ref, dt, m)
    for prec in ("fp64", "mixed"):
        c = Chain(L, J=1.0, alpha=alpha, h=h, prec=prec)
        x = c.new_state()
        c.init_basis_state(x, 0)
        c.krylov_evolve(x, dt, 2, m)
        assert rel(to_host(x), ref) < TOL[prec]
        sz = c.measure_local(x)
        for k in (1, 7, 12, 24):
            want = float(np.real(np.trace(O.SZ @ O.rdm_sites(ref, L, [k]))))
            assert abs(sz[k - 1] - want) < TOL[prec]
        del c, x
        torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# Lanczos steps in three launches (control scalars summed inside the update and
# the next product) against the five-launch sequence
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L", [10, 16, 24])
def test_lanczos_fold_is_bit_identical(L, prec):
    """Krylov evolution (alpha = 1.5, h = 0.8, all-up, m = 20, dt = 0.01, 5 steps) with the
    control kernels folded and not: the same fixed-order sums, so the same bits, also
    for the error estimate."""
    out = []
    for fold in (1, 0):
        c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec=prec)
        c.set_lanczos_fold(fold)
        x = c.new_state()
        c.init_basis_state(x, 0)
        err = c.krylov_evolve(x, 0.01, 5, 20)
        out.append((x.clone(), err))
        c.close()
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lanczos_fold_breakdown_on_an_eigenstate(prec):
    """h = 0: a basis state is an eigenstate, the Krylov space breaks down after one
    vector (the folded test runs in the second product's first pass).  exp(-iE dt)|b>
    for E the diagonal energy, folded and not, bit-identical."""
    L = 14
    b = 0b10110011100101
    res = []
    for fold in (1, 0):
        c = Chain(L, J=1.0, alpha=1.5, h=0.0, prec=prec)
        c.set_lanczos_fold(fold)
        x = c.new_state()
        c.init_basis_state(x, b)
        c.krylov_evolve(x, 0.05, 3, 20)
        res.append(x.clone())
        c.close()
    assert torch.equal(res[0], res[1])
    E = O.diagonal_energy(L, O.coupling_table(L, 1.0, 1.5), np.array([b]))[0]
    got = to_host(res[0])
    ref = np.zeros(1 << L, dtype=np.complex128)
    ref[b] = np.exp(-1j * E * 0.15)
    assert rel(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lanczos_fold_adjoint_bit_identical(prec):
    """The adjoint gradient builds its Krylov bases with the same steps: loss and
    gradient bit-identical with and without the fold (L = 10, 40 steps)."""
    L = 10
    hs = 0.8 + 0.2 * np.sin(np.arange(40) * 0.3)
    res = []
    for fold in (1, 0):
        c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec=prec)
        c.set_lanczos_fold(fold)
        x = c.new_state()
        c.init_basis_state(x, 0)
        res.append(c.adjoint_grad(x, hs, 0.02, m=12))
        c.close()
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1]) and res[0][2] == res[1][2]
