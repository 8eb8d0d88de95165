"""Pins of the FP64 oracle against things other than itself (CPU only).

Each check is chosen so that a plausible slip in the oracle (site order, a
sign, a dropped coupling, a transposed reshape, a wrong Krylov coefficient)
fails at least one of them: hand-typed 2-site matrices, closed forms (free
fermions, Page, J=0 / h=0 dynamics), dense library routines on an
independently built Kronecker Hamiltonian, conservation laws, and numbers the
paper prints.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import seeded_inputs as si
from oracle import ed_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lr_table(L, alpha, J=1.0):
    return np.array([J / r ** alpha for r in range(1, L)])


# --------------------------------------------------------------------------
# Hamiltonian construction
# --------------------------------------------------------------------------

def test_two_site_matrix_by_hand():
    # H = J sz_1 sz_2 + h1 sx_1 + h2 sx_2, basis |s1 s2>, site 1 = high bit.
    J, h1, h2 = 0.7, 0.3, -0.2
    want = np.array([[J, h2, h1, 0.0],
                     [h2, -J, 0.0, h1],
                     [h1, 0.0, -J, h2],
                     [0.0, h1, h2, J]])
    Jr = np.array([J])
    np.testing.assert_array_equal(O.hamiltonian_dense(2, Jr, [h1, h2]), want)
    np.testing.assert_array_equal(O.hamiltonian_csr(2, Jr, [h1, h2]).toarray(), want)


@pytest.mark.parametrize("L", [1, 3, 5, 8])
def test_csr_equals_kronecker(L):
    rng = np.random.default_rng(L)
    Jr = rng.normal(size=L - 1)
    hk = rng.normal(size=L)
    A = O.hamiltonian_csr(L, Jr, hk).toarray()
    B = O.hamiltonian_dense(L, Jr, hk)
    np.testing.assert_allclose(A, B, rtol=0, atol=1e-14)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=0)


def test_ruleset_and_rows_equal_csr():
    L = 11
    Jr = lr_table(L, 1.5)
    psi = si.gaussian_state(L, 7)
    H = O.hamiltonian_csr(L, Jr, 0.8)
    ref = H @ psi
    np.testing.assert_allclose(O.RuleSetH(L, Jr, 0.8)(psi), ref, rtol=0, atol=1e-13)
    rows = np.random.default_rng(0).integers(0, 1 << L, size=300)
    np.testing.assert_allclose(O.apply_H_rows(L, Jr, 0.8, psi, rows), ref[rows], rtol=0, atol=1e-13)


def test_hermiticity():
    L = 10
    Jr = lr_table(L, 0.7, J=-1.3)
    mv = O.RuleSetH(L, Jr, 1.1)
    a, b = si.gaussian_state(L, 1), si.gaussian_state(L, 2)
    assert abs(np.vdot(a, mv(b)) - np.conj(np.vdot(b, mv(a)))) < 1e-13


def test_diagonal_closed_forms():
    # all-up: every pair aligned; Neel: pairs at distance r have sign (-1)^r.
    def up(L, alpha):
        return sum((L - r) / r ** alpha for r in range(1, L))

    def neel(L, alpha):
        return sum((L - r) * (-1) ** r / r ** alpha for r in range(1, L))

    for L, alpha in [(24, 1.5), (20, 2.0), (30, 1.0), (7, 0.0)]:
        Jr = lr_table(L, alpha)
        assert abs(O.diagonal_energy(L, Jr, np.array([0]))[0] - up(L, alpha)) < 1e-12
        nb = si.neel_index(L)
        assert abs(O.diagonal_energy(L, Jr, np.array([nb]))[0] - neel(L, alpha)) < 1e-12
    # values quoted for the three quench workloads
    assert abs(up(24, 1.5) - 44.560736401070486) < 1e-12
    assert abs(up(20, 2.0) - 28.325525221116784) < 1e-12
    assert abs(neel(30, 1.0) - (-20.302744130741935)) < 1e-12


def test_coupling_table_by_hand():
    # J(r) = J / r^alpha typed out by hand (index r-1): 2^-1.5 = 1/(2 sqrt 2),
    # 3^-1.5 = 1/(3 sqrt 3), 4^-1.5 = 1/8; an off-by-one in r or a dropped J fails here
    np.testing.assert_allclose(O.coupling_table(5, 1.0, 1.5),
                               [1.0, 0.35355339059327373, 0.19245008972987526, 0.125], rtol=1e-15, atol=0)
    np.testing.assert_allclose(O.coupling_table(4, -1.3, 2.0), [-1.3, -0.325, -0.14444444444444443],
                               rtol=1e-15, atol=0)
    np.testing.assert_array_equal(O.coupling_table(4, 0.6, 0.0), [0.6, 0.6, 0.6])
    # nearest neighbours only for alpha None or +inf; the table argument overrides both
    np.testing.assert_array_equal(O.coupling_table(4, 2.0, None), [2.0, 0.0, 0.0])
    np.testing.assert_array_equal(O.coupling_table(4, 2.0, math.inf), [2.0, 0.0, 0.0])
    np.testing.assert_array_equal(O.coupling_table(3, 1.0, 1.5, table=[0.1, -0.2]), [0.1, -0.2])
    assert O.coupling_table(1, 1.0, 1.5).shape == (0,)
    # the all-up diagonal energy sum_r (L - r) J(r) of the L = 24, alpha = 1.5 quench,
    # through coupling_table and through the oracle's pair loop, against the typed value
    Jr = O.coupling_table(24, 1.0, 1.5)
    assert abs(sum((24 - r) * Jr[r - 1] for r in range(1, 24)) - 44.560736401070486) < 1e-12
    assert abs(O.diagonal_energy(24, Jr, np.array([0]))[0] - 44.560736401070486) < 1e-12
    Jr = O.coupling_table(30, 1.0, 1.0)
    assert abs(O.diagonal_energy(30, Jr, np.array([si.neel_index(30)]))[0] - (-20.302744130741935)) < 1e-12


# --------------------------------------------------------------------------
# Ground state
# --------------------------------------------------------------------------

def test_jordan_wigner_vs_csc_closed_form():
    # uniform J = h = 1: E0 = 1 - csc(pi / (2 (2L + 1))) (Pfeuty 1970)
    for L in (2, 6, 12):
        want = 1.0 - 1.0 / math.sin(math.pi / (2 * (2 * L + 1)))
        assert abs(O.jordan_wigner_ground_energy(L, 1.0, 1.0) - want) < 1e-12


def test_lanczos_matches_free_fermions_L12():
    L = 12
    Jr = O.coupling_table(L, J=-1.0, alpha=None)  # Eq. HQI sign convention
    H = O.hamiltonian_csr(L, Jr, -1.0)
    x0 = si.gaussian_state(L, 1)
    E, x, res, it = O.lanczos_ground(O.csr_matvec(H), x0, tol=1e-12, max_iter=400)
    assert abs(E - (-14.925971109908655)) < 1e-11
    assert res <= 1e-12
    # the sign convention of J and h does not change the NN spectrum
    H2 = O.hamiltonian_csr(L, -Jr, 1.0)
    E2, _, _, _ = O.lanczos_ground(O.csr_matvec(H2), x0, tol=1e-12, max_iter=400)
    assert abs(E2 - E) < 1e-11


@pytest.mark.parametrize("L,alpha,h,J", [(8, 1.5, 0.8, 1.0), (9, 0.5, 0.3, -1.0), (10, 3.0, 1.7, 1.0)])
def test_lanczos_matches_dense_eigh(L, alpha, h, J):
    Jr = lr_table(L, alpha, J)
    Hd = O.hamiltonian_dense(L, Jr, h)
    e = np.linalg.eigvalsh(Hd)
    E, x, res, it = O.lanczos_ground(lambda v: Hd @ v, si.gaussian_state(L, 3), tol=1e-10, max_iter=500)
    assert E >= e[0] - 1e-10
    assert abs(E - e[0]) < 1e-9


def test_pure_field_ground_energy():
    L = 9
    hk = np.linspace(-1.0, 1.5, L)
    H = O.hamiltonian_csr(L, np.zeros(L - 1), hk)
    E, _, _, _ = O.lanczos_ground(O.csr_matvec(H), si.gaussian_state(L, 5), tol=1e-11)
    assert abs(E + np.sum(np.abs(hk))) < 1e-10


# --------------------------------------------------------------------------
# Krylov time step
# --------------------------------------------------------------------------

def test_krylov_matches_dense_expm():
    L = 8
    Jr = lr_table(L, 1.5)
    Hd = O.hamiltonian_dense(L, Jr, 0.8)
    psi = si.gaussian_state(L, 11)
    out = psi.copy()
    for _ in range(10):
        out, err = O.krylov_step(lambda v: Hd @ v, out, 0.05, 20)
    want = sla.expm(-1j * 0.5 * Hd) @ psi
    assert np.linalg.norm(out - want) < 1e-12


def test_krylov_exact_when_space_exhausted():
    # paper: Krylov is exact for time-independent H regardless of dt
    L = 3
    Hd = O.hamiltonian_dense(L, lr_table(L, 1.0), 0.9)
    psi = si.gaussian_state(L, 2)
    out, _ = O.krylov_step(lambda v: Hd @ v, psi, 2.5, 1 << L)
    want = sla.expm(-1j * 2.5 * Hd) @ psi
    assert np.linalg.norm(out - want) < 1e-12


def test_pure_field_quench_closed_form():
    # J = 0 from all-up: <sz_i(t)> = cos(2ht), <sz_i sz_j> = cos(2ht)^2, S = 0
    L, h, dt = 10, 0.7, 0.1
    H = O.hamiltonian_csr(L, np.zeros(L - 1), h)
    psi = si.basis_state(L, 0)
    t = 0.0
    for _ in range(13):
        psi, _ = O.krylov_step(O.csr_matvec(H), psi, dt, 12)  # breaks down at L+1 vectors
        t += dt
    c = math.cos(2 * h * t)
    np.testing.assert_allclose(O.measure_local(psi, L), c, atol=1e-12)
    C = O.measure_corr(psi, L)
    off = C[~np.eye(L, dtype=bool)]
    np.testing.assert_allclose(off, c * c, atol=1e-12)
    assert abs(O.schmidt_entropy(psi, L)) < 1e-10


def test_zero_field_phases():
    # h = 0: psi_b(t) = exp(-i E(b) t) psi_b
    L = 8
    Jr = lr_table(L, 1.2)
    mv = O.RuleSetH(L, Jr, 0.0)
    psi = si.gaussian_state(L, 4)
    out = psi.copy()
    for _ in range(20):
        out, _ = O.krylov_step(mv, out, 0.02, 25)
    E = np.array([sum(Jr[j - i - 1] * (1 - 2 * ((b >> (L - i)) & 1)) * (1 - 2 * ((b >> (L - j)) & 1))
                      for i in range(1, L + 1) for j in range(i + 1, L + 1)) for b in range(1 << L)])
    np.testing.assert_allclose(out, np.exp(-1j * E * 0.4) * psi, atol=1e-11)


def test_conservation_laws():
    L = 10
    Jr = lr_table(L, 1.5)
    mv = O.RuleSetH(L, Jr, 0.8)
    psi = si.gaussian_state(L, 9)
    flip = (1 << L) - 1
    idx = np.arange(1 << L)

    def parity(v):
        return np.vdot(v, v[idx ^ flip])

    n0, e0, p0 = np.linalg.norm(psi), O.energy(mv, psi), parity(psi)
    out = psi
    for _ in range(20):
        out, _ = O.krylov_step(mv, out, 0.05, 20)
    assert abs(np.linalg.norm(out) - n0) < 1e-12
    assert abs(O.energy(mv, out) - e0) < 1e-10
    assert abs(parity(out) - p0) < 1e-11


def test_midpoint_rate_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["ising_linear_quench_rates"]
    L = g["L"]
    Jr = O.coupling_table(L, J=-1.0, alpha=None)
    Hzz = O.hamiltonian_csr(L, Jr, 0.0)
    Hx = O.hamiltonian_csr(L, np.zeros(L - 1), -1.0)
    e, v = np.linalg.eigh((Hzz + g["h_start"] * Hx).toarray())
    psi0 = v[:, 0].astype(np.complex128)

    def hfun(t):
        return g["h_start"] + (g["h_end"] - g["h_start"]) * t / g["t_end"]

    def run(dt):
        n = int(round(g["t_end"] / dt))
        return O.evolve(lambda hv: (lambda x, H=(Hzz + hv * Hx): H @ x), psi0, dt, n, 25, field_at=hfun)

    ref = run(g["dt_ref"])
    e1 = O.eps_local(run(0.1), ref, L)
    e2 = O.eps_local(run(0.01), ref, L)
    r = O.convergence_rate(e1, e2, 10.0)
    assert abs(r - g["krylov_rate_dt_0.1_vs_0.01"]) < 0.1, r


# --------------------------------------------------------------------------
# Measurements and entropy
# --------------------------------------------------------------------------

def test_product_and_ghz_measurements():
    L = 9
    up = si.basis_state(L, 0)
    np.testing.assert_allclose(O.measure_local(up, L), 1.0)
    neel = si.basis_state(L, si.neel_index(L))
    np.testing.assert_allclose(O.measure_local(neel, L), [(-1) ** k for k in range(L)])
    C = O.measure_corr(neel, L)
    np.testing.assert_allclose(C, [[(-1) ** (i + j) for j in range(L)] for i in range(L)])
    assert O.schmidt_entropy(neel, L) == 0.0
    ghz = si.ghz_state(L)
    np.testing.assert_allclose(O.measure_local(ghz, L), 0.0, atol=1e-15)
    np.testing.assert_allclose(O.measure_corr(ghz, L), 1.0, atol=1e-15)
    assert abs(O.schmidt_entropy(ghz, L) - math.log(2.0)) < 1e-14


def test_rdm_route_equals_brute_force():
    L = 8
    psi = si.gaussian_state(L, 21)
    p = np.abs(psi) ** 2
    b = np.arange(1 << L)
    s = [1 - 2 * ((b >> (L - k)) & 1) for k in range(1, L + 1)]
    np.testing.assert_allclose(O.measure_local(psi, L), [np.sum(p * s[k]) for k in range(L)], atol=1e-14)
    C = O.measure_corr(psi, L)
    want = np.array([[np.sum(p * s[i] * s[j]) for j in range(L)] for i in range(L)])
    np.testing.assert_allclose(C, want, atol=1e-14)
    assert abs(O.measure_corr_pair(psi, L, 2, 7) - want[1, 6]) < 1e-14


def test_schmidt_spectrum_invariants_and_svd():
    for L in (7, 10):
        psi = si.gaussian_state(L, L) * 1.3
        lam = O.schmidt_spectrum(psi, L)
        l = L // 2
        M = psi.reshape(1 << l, 1 << (L - l))
        sv = np.linalg.svd(M, compute_uv=False) ** 2
        np.testing.assert_allclose(lam, np.sort(sv)[::-1], atol=1e-13)
        assert abs(np.sum(lam) - np.vdot(psi, psi).real) < 1e-12
        assert np.all(lam > -1e-14)
        right = np.sort(np.linalg.eigvalsh(M.conj().T @ M))[::-1][: len(lam)]
        np.testing.assert_allclose(lam, right, atol=1e-13)


def test_schmidt_spectrum_small_side_equals_singular_values():
    """Both branches (left block smaller / larger) against the squared singular
    values of M, which a plain SVD fixes independently of either Gram matrix."""
    L = 9
    psi = si.gaussian_state(L, 44)
    for l in (1, 3, 4, 5, 8):
        M = psi.reshape(1 << l, 1 << (L - l))
        sv = np.sort(np.linalg.svd(M, compute_uv=False) ** 2)[::-1]
        lam = O.schmidt_spectrum_small(psi, L, l)
        assert len(lam) == 1 << min(l, L - l)
        np.testing.assert_allclose(lam, sv, atol=1e-13)


def test_page_value():
    # Haar-random state, equal bipartition m = n: Page (1993) mean entropy.
    L = 14
    m = n = 1 << (L // 2)
    page = sum(1.0 / k for k in range(n + 1, m * n + 1)) - (m - 1) / (2.0 * n)
    vals = [O.schmidt_entropy(si.gaussian_state(L, s), L) for s in range(3)]
    assert abs(np.mean(vals) - page) < 5e-3


def test_trace_distance_and_rate_helpers():
    r1 = np.diag([1.0, 0.0])
    r2 = np.diag([0.0, 1.0])
    assert abs(O.trace_distance(r1, r2) - 1.0) < 1e-15
    assert abs(O.convergence_rate(1e-2, 1e-4, 10.0) - 2.0) < 1e-12


# ---------------------------------------------------------------------------
# ground_energy_sparse (reference energies of the batched ground states)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L,alpha,h", [(8, 0.5, 0.2), (9, 2.5, 1.8), (10, 1.3, 0.7)])
def test_sparse_ground_energy_matches_dense_eigh(L, alpha, h):
    """eigsh on the entry-by-entry CSR matrix against dense eigh of the
    Kronecker-product Hamiltonian (two independent constructions)."""
    Jr = O.coupling_table(L, 1.0, alpha)
    E_dense = float(np.linalg.eigvalsh(O.hamiltonian_dense(L, Jr, h))[0])
    assert abs(O.ground_energy_sparse(L, Jr, h) - E_dense) < 1e-11 * max(1.0, abs(E_dense))


@pytest.mark.parametrize("L,h", [(13, 1.0), (14, 0.4)])
def test_sparse_ground_energy_matches_jordan_wigner(L, h):
    """Nearest-neighbour chains beyond dense size: the free-fermion closed form."""
    Jr = O.coupling_table(L, 1.0, None)
    E_jw = O.jordan_wigner_ground_energy(L, 1.0, h)
    assert abs(O.ground_energy_sparse(L, Jr, h) - E_jw) < 1e-11 * abs(E_jw)


# ---------------------------------------------------------------------------
# final_energy_gradient_dense (reference gradients of the adjoint sweep)
# ---------------------------------------------------------------------------

def _fe_case(L=4, n=6, seed=41):
    rng = np.random.Generator(np.random.Philox(seed))
    return L, O.coupling_table(L, 1.0, 2.0), rng.uniform(0.5, 1.5, size=n), 0.07, si.basis_state(L, 0)


def test_final_energy_gradient_matches_central_differences():
    """Block-exponential (Frechet) gradients against central differences of the dense
    expm forward model (a different path to the same derivative)."""
    L, Jr, hs, dt, psi0 = _fe_case()
    loss, gh, gs = O.final_energy_gradient_dense(L, Jr, hs, dt, 1.0, psi0)
    eps = 1e-6
    for k in range(len(hs)):
        hp, hm = hs.copy(), hs.copy()
        hp[k] += eps
        hm[k] -= eps
        fd = (O.final_energy_gradient_dense(L, Jr, hp, dt, 1.0, psi0)[0]
              - O.final_energy_gradient_dense(L, Jr, hm, dt, 1.0, psi0)[0]) / (2 * eps)
        assert abs(fd - gh[k]) < 1e-7 * max(1.0, abs(gh[k]))
    fd = (O.final_energy_gradient_dense(L, (1 + eps) * Jr, hs, dt, 1.0, psi0)[0]
          - O.final_energy_gradient_dense(L, (1 - eps) * Jr, hs, dt, 1.0, psi0)[0]) / (2 * eps)
    assert abs(fd - gs) < 1e-7 * max(1.0, abs(gs))


def test_final_energy_gradient_zero_field_closed_form():
    """h_k = 0: the all-up state only acquires a phase, so loss = <up|H_zz|up> and
    dloss/ds = sum_r (L - r) J(r) exactly."""
    L = 5
    Jr = O.coupling_table(L, 1.0, 1.5)
    loss, gh, gs = O.final_energy_gradient_dense(L, Jr, np.zeros(4), 0.1, 1.0, si.basis_state(L, 0))
    want = sum((L - r) * Jr[r - 1] for r in range(1, L))
    assert abs(loss - want) < 1e-12 and abs(gs - want) < 1e-11


def test_final_energy_krylov_matches_dense_loss():
    L, Jr, hs, dt, psi0 = _fe_case(L=5, n=4, seed=43)
    dense = O.final_energy_gradient_dense(L, Jr, hs, dt, 1.0, psi0)[0]
    assert abs(O.final_energy_krylov(L, Jr, hs, dt, 20, 1.0, psi0) - dense) < 1e-11 * max(1.0, abs(dense))


# ---------------------------------------------------------------------------
# Trotter decomposition and two-site gates (Sec. III.C, App. C)
# ---------------------------------------------------------------------------

def test_two_site_contraction_matches_kronecker_embedding():
    L = 5
    rng = np.random.Generator(np.random.Philox(51))
    psi = si.gaussian_state(L, 52)
    U = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    for s in range(1, L):
        full = np.kron(np.kron(np.eye(1 << (s - 1)), U), np.eye(1 << (L - s - 1)))
        np.testing.assert_allclose(O.apply_two_site(psi, L, s, U), full @ psi, atol=1e-13)


@pytest.mark.parametrize("order", [1, 2, 4])
def test_trotter_tensor_matches_dense_layers(order):
    L = 6
    psi = si.gaussian_state(L, 53)
    a = O.trotter_evolve_tensor(psi, L, 1.0, 0.7, 0.1, 3, order)
    b = O.trotter_evolve_dense(psi, L, 1.0, 0.7, 0.1, 3, order)
    assert np.linalg.norm(a - b) < 1e-12


def test_trotter_sum_of_layers_is_the_hamiltonian():
    """sum of bond terms with the 1/2 (1 at the ends) site weights = H of Eq. HQI."""
    L = 6
    terms = O.bond_terms(L, -1.0, -0.8)
    H = sum(np.kron(np.kron(np.eye(1 << (s - 1)), t), np.eye(1 << (L - s - 1))) for s, t in terms.items())
    np.testing.assert_allclose(H, O.hamiltonian_dense(L, O.coupling_table(L, -1.0, None), -0.8), atol=1e-13)


def test_trotter_exact_without_bonds():
    """J = 0: all layer terms commute, so every order is exact."""
    L = 6
    psi = si.gaussian_state(L, 54)
    exact = O.exact_propagate_dense(O.hamiltonian_dense(L, O.coupling_table(L, 0.0, None), 0.9), psi, 0.5)
    for order in (1, 2, 4):
        assert np.linalg.norm(O.trotter_evolve_tensor(psi, L, 0.0, 0.9, 0.1, 5, order) - exact) < 1e-12


@pytest.mark.parametrize("order,rate", [(1, 1.0), (2, 2.0), (4, 4.0)])
def test_trotter_convergence_order(order, rate):
    """Global error at fixed t falls like dt^order (Sec. V convergence studies)."""
    L, t = 8, 0.8
    psi = si.gaussian_state(L, 55)
    exact = O.exact_propagate_dense(O.hamiltonian_dense(L, O.coupling_table(L, 1.0, None), 0.6), psi, t)
    errs = []
    for n in (8, 16):
        errs.append(np.linalg.norm(O.trotter_evolve_tensor(psi, L, 1.0, 0.6, t / n, n, order) - exact))
    assert abs(math.log2(errs[0] / errs[1]) - rate) < 0.25


# ---------------------------------------------------------------------------
# two-site reduced density matrices (references of the all-pairs RDM kernel)
# ---------------------------------------------------------------------------

def test_pair_rdm_closed_forms():
    """Product state: rho_ij = |a_i><a_i| (x) |a_j><a_j|; GHZ: (|00><00| + |11><11|)/2;
    a Bell pair on sites (2, 4) of a product state: the Bell projector."""
    L = 5
    b = si.neel_index(L)
    psi = si.basis_state(L, b)
    bits = [(b >> (L - s)) & 1 for s in range(1, L + 1)]
    for i, j in ((1, 2), (2, 5), (3, 4)):
        want = np.zeros((4, 4))
        v = 2 * bits[i - 1] + bits[j - 1]
        want[v, v] = 1.0
        np.testing.assert_allclose(O.rdm_sites(psi, L, (i, j)), want, atol=1e-15)
    g = si.ghz_state(L)
    np.testing.assert_allclose(O.rdm_sites(g, L, (1, 4)), np.diag([0.5, 0, 0, 0.5]), atol=1e-15)
    bell = np.zeros(1 << L, dtype=np.complex128)
    bell[0] = 1 / math.sqrt(2)                               # sites 2, 4 both up
    bell[(1 << (L - 2)) | (1 << (L - 4))] = 1j / math.sqrt(2)  # sites 2, 4 both down
    want = np.zeros((4, 4), dtype=np.complex128)
    want[0, 0] = want[3, 3] = 0.5
    want[0, 3] = -0.5j
    want[3, 0] = 0.5j
    np.testing.assert_allclose(O.rdm_sites(bell, L, (2, 4)), want, atol=1e-15)


def test_pair_rdm_partial_trace_and_positivity():
    L = 6
    psi = si.gaussian_state(L, 81)
    r = O.rdm_sites(psi, L, (2, 5))
    assert abs(np.trace(r) - 1.0) < 1e-13
    np.testing.assert_allclose(r, r.conj().T, atol=1e-15)
    assert np.linalg.eigvalsh(r).min() > -1e-14
    tr_j = r.reshape(2, 2, 2, 2).trace(axis1=1, axis2=3)
    np.testing.assert_allclose(tr_j, O.rdm_sites(psi, L, (2,)), atol=1e-14)
