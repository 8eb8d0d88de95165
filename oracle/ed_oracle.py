"""Plain FP64 CPU oracle for the exact-diagonalization hot path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
the CPU-baseline leg of the benchmark may import this module.  The GPU library
never calls it, and it shares no code with the GPU library: the only common
dependency is the seeded input generator module, which holds no arithmetic of
the method.

Everything here is deliberately slow and obvious, in float64 / complex128:

* the Hamiltonian built entry by entry from its definition (sparse CSR), and
  independently by Kronecker products of Pauli matrices (dense, small L);
* a rule-set times state product on the rank-L tensor view of psi, the
  matrix-free route the paper uses beyond twenty qubits (Sec. III.D);
* Lanczos ground state with full reorthogonalisation;
* one Krylov step exp(-i H dt) psi with the basis orthogonalised against all
  previous vectors and the small exponential taken in the Krylov basis
  (Sec. III.D, Krylov approximation);
* measurements through reduced density matrices (Sec. IV) and the bond
  entropy through rho = M M^dagger (Sec. IV, bond entropy).

Model (Eq. genericH restricted to one site rule and one distance-only
infinite-function rule; Eq. HQI and the long-range H_LRQI of Sec. VII are the
special cases J(r) = -delta_{r,1}, h -> -h and J(r) = -cos(phi)/r^alpha,
h = -sin(phi)):

    H = sum_{i<j} J(j-i) sz_i sz_j + sum_k h_k sx_k

with signed inputs.  Site k (1-based) is bit L-k of the basis index b (site 1
is the most significant bit, the paper's row-major rank-L tensor); bit value 0
is spin up, sz = +1.

Pins: every function here is checked in tests/test_oracle_pins.py against
things other than itself (Jordan-Wigner closed form, dense eigh / expm of the
Kronecker Hamiltonian, analytic J=0 and h=0 dynamics, conservation laws,
product / GHZ / Page states, SVD).  No function is parity-unpinned.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

SX = np.array([[0.0, 1.0], [1.0, 0.0]])
SZ = np.array([[1.0, 0.0], [0.0, -1.0]])
I2 = np.eye(2)


# ---------------------------------------------------------------------------
# Couplings and fields
# ---------------------------------------------------------------------------

def coupling_table(L: int, J: float = 1.0, alpha=None, table=None) -> np.ndarray:
    """Distance-only coupling J(r) for r = 1..L-1 (returned with index r-1).

    The infinite-function rule couples sites k < k' with c(k'-k) that depends
    only on the distance (Eq. genericH, long-range term; App. A).  ``alpha``
    None (or inf) keeps nearest neighbours only: J(1) = J, J(r>1) = 0.
    Otherwise J(r) = J / r^alpha.  ``table`` overrides both.
    """
    if table is not None:
        t = np.asarray(table, dtype=np.float64)
        assert t.shape == (max(L - 1, 0),)
        return t.copy()
    r = np.arange(1, L, dtype=np.float64)
    if alpha is None or (isinstance(alpha, float) and math.isinf(alpha)):
        out = np.zeros(max(L - 1, 0))
        if L > 1:
            out[0] = J
        return out
    return J / r ** float(alpha)


def site_fields(L: int, h) -> np.ndarray:
    """Transverse field h_k per site k = 1..L (index k-1); a scalar is uniform."""
    hk = np.asarray(h, dtype=np.float64)
    if hk.ndim == 0:
        return np.full(L, float(hk))
    assert hk.shape == (L,)
    return hk.copy()


def sz_of(L: int, b: np.ndarray, k: int) -> np.ndarray:
    """sigma^z eigenvalue of site k (1-based) in basis states b."""
    return 1 - 2 * ((b >> (L - k)) & 1)


# ---------------------------------------------------------------------------
# Hamiltonian: definition, Kronecker construction, CSR
# ---------------------------------------------------------------------------

def diagonal_energy(L: int, Jr: np.ndarray, b: np.ndarray) -> np.ndarray:
    """E(b) = sum_{i<j} J(j-i) s_i(b) s_j(b): the plain O(L^2) pair loop."""
    b = np.asarray(b, dtype=np.int64)
    E = np.zeros(b.shape, dtype=np.float64)
    for i in range(1, L + 1):
        si = sz_of(L, b, i)
        for j in range(i + 1, L + 1):
            E += Jr[j - i - 1] * si * sz_of(L, b, j)
    return E


def _site_op(L: int, k: int, op: np.ndarray) -> np.ndarray:
    """op on site k padded with identities by Kronecker products (site 1 leftmost)."""
    left = np.eye(1 << (k - 1))
    right = np.eye(1 << (L - k))
    return np.kron(np.kron(left, op), right)


def hamiltonian_dense(L: int, Jr: np.ndarray, h) -> np.ndarray:
    """Dense H from Kronecker products of Pauli matrices (Sec. II, Eq. OH route)."""
    hk = site_fields(L, h)
    D = 1 << L
    H = np.zeros((D, D))
    Z = [_site_op(L, k, SZ) for k in range(1, L + 1)]
    for i in range(1, L + 1):
        for j in range(i + 1, L + 1):
            H += Jr[j - i - 1] * (Z[i - 1] @ Z[j - 1])
        H += hk[i - 1] * _site_op(L, i, SX)
    return H


def hamiltonian_csr(L: int, Jr: np.ndarray, h) -> sp.csr_matrix:
    """H as an explicit FP64 CSR matrix, entry by entry from the definition.

    Row b holds the diagonal E(b) and one entry h_k at column b XOR 2^(L-k)
    for every site k: L+1 non-zeros per row.
    """
    hk = site_fields(L, h)
    D = 1 << L
    rows = np.arange(D, dtype=np.int64)
    r_list = [rows]
    c_list = [rows]
    d_list = [diagonal_energy(L, Jr, rows)]
    for k in range(1, L + 1):
        r_list.append(rows)
        c_list.append(rows ^ (1 << (L - k)))
        d_list.append(np.full(D, hk[k - 1]))
    H = sp.coo_matrix((np.concatenate(d_list), (np.concatenate(r_list), np.concatenate(c_list))),
                      shape=(D, D)).tocsr()
    H.sum_duplicates()
    return H


def apply_H_rows(L: int, Jr: np.ndarray, h, psi: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """(H psi)_b for a chosen set of rows b, straight from the definition.

    Uses the O(L^2) pair loop for the diagonal and one gather per site for the
    flips, so any row of a large chain can be checked without building H.
    """
    hk = site_fields(L, h)
    rows = np.asarray(rows, dtype=np.int64)
    out = diagonal_energy(L, Jr, rows) * psi[rows]
    for k in range(1, L + 1):
        out = out + hk[k - 1] * psi[rows ^ (1 << (L - k))]
    return out


class RuleSetH:
    """Matrix-free H psi on the rank-L tensor view of psi (Sec. III.D, mode 2).

    The diagonal E(b) is tabulated once with the pair loop; each sigma^x_k acts
    by reversing axis k-1 of the (2,)*L tensor, the tensordot-with-sigma^x of
    the rule-set times state product.
    """

    def __init__(self, L: int, Jr: np.ndarray, h):
        self.L = L
        self.Jr = np.asarray(Jr, dtype=np.float64)
        self.hk = site_fields(L, h)
        self.E = diagonal_energy(L, self.Jr, np.arange(1 << L, dtype=np.int64))

    def set_field(self, h):
        self.hk = site_fields(self.L, h)

    def __call__(self, psi: np.ndarray) -> np.ndarray:
        L = self.L
        out = self.E * psi
        T = psi.reshape((2,) * L) if L > 0 else psi
        acc = out.reshape((2,) * L) if L > 0 else out
        for k in range(1, L + 1):
            if self.hk[k - 1] != 0.0:
                acc += self.hk[k - 1] * np.flip(T, axis=k - 1)
        return acc.reshape(-1)


def csr_matvec(H: sp.csr_matrix):
    return lambda x: H @ x


# ---------------------------------------------------------------------------
# Closed forms used as pins (not used by any other oracle function)
# ---------------------------------------------------------------------------

def jordan_wigner_ground_energy(L: int, J: float, h: float) -> float:
    """Ground energy of the open chain H = -J sum sz sz - h sum sx.

    Free-fermion solution (Lieb-Schultz-Mattis 1961, Pfeuty 1970): minus the
    sum of the singular values of the L x L upper-bidiagonal matrix with h on
    the diagonal and J on the super-diagonal.  The sign of J or h does not
    change the spectrum of the nearest-neighbour chain.
    """
    B = np.diag(np.full(L, abs(h))) + np.diag(np.full(L - 1, abs(J)), 1)
    return -float(np.sum(np.linalg.svd(B, compute_uv=False)))


def ground_energy_sparse(L: int, Jr: np.ndarray, h) -> float:
    """Lowest eigenvalue of the CSR Hamiltonian by ARPACK (scipy eigsh, the
    routine the paper uses for statics, Sec. II): the plain definition of the
    ground energy for chains too long for dense eigh."""
    from scipy.sparse.linalg import eigsh

    H = hamiltonian_csr(L, Jr, h)
    # a generic start vector: a symmetric one (e.g. all ones) stays inside one
    # parity / reflection sector and can miss the ground state
    v0 = np.random.Generator(np.random.Philox(20180227)).standard_normal(H.shape[0])
    vals = eigsh(H, k=1, which="SA", tol=1e-13, v0=v0, return_eigenvectors=False)
    return float(vals[0])


# ---------------------------------------------------------------------------
# Small tridiagonal helpers (library routines as steps)
# ---------------------------------------------------------------------------

def _tridiag(alpha, beta) -> np.ndarray:
    m = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=np.float64))
    if m > 1:
        T += np.diag(np.asarray(beta[: m - 1], dtype=np.float64), 1)
        T += np.diag(np.asarray(beta[: m - 1], dtype=np.float64), -1)
    return T


# ---------------------------------------------------------------------------
# Lanczos ground state (statics, Sec. II; eigsh replaced by an explicit
# Lanczos with full reorthogonalisation)
# ---------------------------------------------------------------------------

def lanczos_ground(matvec, x0: np.ndarray, tol: float = 1e-12, max_iter: int = 300):
    """Lowest eigenpair of a Hermitian operator by Lanczos with full reorth.

    Stops when the explicit residual ||H x - theta x|| <= tol for the
    normalised Ritz vector x (checked whenever the estimate
    beta_{j+1} |y_j| drops below tol, or on breakdown, or at max_iter).
    Returns (theta, x, residual, iterations).
    """
    V = [x0 / np.linalg.norm(x0)]
    alpha, beta = [], []
    theta, x, res = None, None, None
    for j in range(max_iter):
        w = matvec(V[j])
        a = float(np.real(np.vdot(V[j], w)))
        w = w - a * V[j]
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        for _ in range(2):  # full reorthogonalisation, twice
            for v in V:
                w = w - np.vdot(v, w) * v
        alpha.append(a)
        b = float(np.linalg.norm(w))
        beta.append(b)
        evals, evecs = np.linalg.eigh(_tridiag(alpha, beta))
        theta = float(evals[0])
        y = evecs[:, 0]
        est = b * abs(y[-1])
        done = est <= tol or b < 1e-300 or j == max_iter - 1 or len(V) == len(x0)
        if done or est <= 10 * tol:
            x = np.zeros_like(V[0])
            for i, v in enumerate(V):
                x = x + y[i] * v
            x /= np.linalg.norm(x)
            res = float(np.linalg.norm(matvec(x) - theta * x))
            if res <= tol or done:
                return theta, x, res, j + 1
        V.append(w / b)
    return theta, x, res, max_iter


# ---------------------------------------------------------------------------
# Krylov time step (Sec. III.D)
# ---------------------------------------------------------------------------

def krylov_step(matvec, psi: np.ndarray, dt: float, m: int, breakdown: float = 1e-14):
    """psi(t+dt) ~ sum_i xi_i v_i with xi_i = ||psi|| [exp(-i dt T_m)]_{i,1}.

    v_1 = psi/||psi||; v_{i+1} is H v_i orthogonalised against all previous
    v_j (twice, classical Gram-Schmidt); T_m holds the projections
    <v_i|H|v_j>, tridiagonal for Hermitian H.  A basis vector whose norm falls
    below ``breakdown``*||psi|| ends the basis early (the subspace is then
    invariant and the step exact).  Returns (psi_new, err_estimate) where the
    estimate is beta_{m+1} |xi_m| (Saad 1992).
    """
    nrm = float(np.linalg.norm(psi))
    V = [psi / nrm]
    alpha, beta = [], []
    for j in range(m):
        w = matvec(V[j])
        a = float(np.real(np.vdot(V[j], w)))
        w = w - a * V[j]
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        for _ in range(2):
            for v in V:
                w = w - np.vdot(v, w) * v
        alpha.append(a)
        b = float(np.linalg.norm(w))
        beta.append(b)
        if b < breakdown:
            break
        if j < m - 1:
            V.append(w / b)
    k = len(alpha)
    T = _tridiag(alpha, beta)
    U = sla.expm(-1j * dt * T)
    xi = nrm * U[:, 0]
    out = np.zeros_like(psi, dtype=np.complex128)
    for i in range(min(k, len(V))):
        out = out + xi[i] * V[i]
    err = beta[k - 1] * abs(xi[k - 1])
    return out, float(err)


def evolve(make_matvec, psi0: np.ndarray, dt: float, nsteps: int, m: int, field_at=None,
           t0: float = 0.0, callback=None):
    """Krylov propagation over nsteps steps of dt.

    ``make_matvec(h)`` returns H(h) psi; ``field_at(t)`` gives the field at
    time t and is evaluated at mid-step t + dt/2 (Sec. III.A, couplings taken
    at the middle of the step).  ``callback(step, t, psi)`` runs after each
    step.
    """
    psi = psi0.astype(np.complex128)
    t = t0
    mv = make_matvec(None) if field_at is None else None
    for s in range(nsteps):
        if field_at is not None:
            mv = make_matvec(field_at(t + 0.5 * dt))
        psi, _ = krylov_step(mv, psi, dt, m)
        t += dt
        if callback is not None:
            callback(s + 1, t, psi)
    return psi


# ---------------------------------------------------------------------------
# Trotter decomposition for nearest-neighbour chains (Sec. III.C) and
# two-site gates on the rank-L tensor (Fig. of the tensor operations; App. C)
# ---------------------------------------------------------------------------

def apply_two_site(psi: np.ndarray, L: int, site: int, U: np.ndarray) -> np.ndarray:
    """Contract a 4 x 4 operator (basis index 2 sigma_s + sigma_{s+1}) with the two
    indices of sites (s, s+1) of psi viewed as a rank-L tensor (site 1 first),
    the tensordot route of Sec. III.C."""
    T = np.asarray(psi, dtype=np.complex128).reshape((2,) * L)
    G = np.asarray(U, dtype=np.complex128).reshape(2, 2, 2, 2)  # (out_s, out_s1, in_s, in_s1)
    T = np.tensordot(G, T, axes=([2, 3], [site - 1, site]))  # new axes 0, 1 = sites s, s+1 first
    T = np.moveaxis(T, [0, 1], [site - 1, site])
    return T.reshape(-1)


def bond_terms(L: int, J1: float, h):
    """Two-site terms h_(s,s+1) = J1 sz sz + w_s h_s sx(x)1 + w_{s+1} h_{s+1} 1(x)sx with site
    weights 1/2 (1 for the first and last site): H = sum_s h_(s,s+1) (Sec. III.C)."""
    hk = site_fields(L, h)
    terms = {}
    for s in range(1, L):
        ws = 1.0 if s == 1 else 0.5
        ws1 = 1.0 if s + 1 == L else 0.5
        terms[s] = J1 * np.kron(SZ, SZ) + ws * hk[s - 1] * np.kron(SX, I2) + ws1 * hk[s] * np.kron(I2, SX)
    return terms


def trotter_factors(order: int):
    """(parity, fraction of dt) of the layers of one step, applied first to last:
    parity 0 = H_e (bonds from even sites), 1 = H_o.  Eqs. trotter1, trotter2, trotter4/4c."""
    if order == 1:
        return [(0, 1.0), (1, 1.0)]
    if order == 2:
        return [(0, 0.5), (1, 1.0), (0, 0.5)]
    t3 = 1.0 / (2.0 * (4.0 - 4.0 ** (1.0 / 3.0)))
    t1, t2, t4 = 1.0 - 8.0 * t3, 0.5 * (1.0 - 6.0 * t3), 2.0 * t3
    seq = [t3, t4, t4, t4, t2, t1, t2, t4, t4, t4, t3]
    return [(1 if f % 2 else 0, x) for f, x in enumerate(seq)]


def trotter_evolve_tensor(psi: np.ndarray, L: int, J1: float, h, dt: float, nsteps: int, order: int) -> np.ndarray:
    """Trotter evolution by two-site propagators expm(-i tau h_bond) applied on the tensor."""
    terms = bond_terms(L, J1, h)
    psi = np.asarray(psi, dtype=np.complex128)
    cache = {}
    for _ in range(nsteps):
        for parity, frac in trotter_factors(order):
            for s in range(1, L):
                if s % 2 != parity:
                    continue
                key = (s, frac)
                if key not in cache:
                    cache[key] = sla.expm(-1j * frac * dt * terms[s])
                psi = apply_two_site(psi, L, s, cache[key])
    return psi


def trotter_evolve_dense(psi: np.ndarray, L: int, J1: float, h, dt: float, nsteps: int, order: int) -> np.ndarray:
    """The same product from the dense layer Hamiltonians H_o, H_e built by Kronecker
    products (small L)."""
    terms = bond_terms(L, J1, h)
    D = 1 << L
    Hp = [np.zeros((D, D)), np.zeros((D, D))]
    for s, t in terms.items():
        Hp[s % 2] += np.kron(np.kron(np.eye(1 << (s - 1)), t), np.eye(1 << (L - s - 1)))
    psi = np.asarray(psi, dtype=np.complex128)
    for _ in range(nsteps):
        for parity, frac in trotter_factors(order):
            psi = sla.expm(-1j * frac * dt * Hp[parity]) @ psi
    return psi


# ---------------------------------------------------------------------------
# Gradient of a final energy under a piecewise-constant field (the paper has
# no gradients: the derivative of its Krylov/expm time evolution, Sec. III.D)
# ---------------------------------------------------------------------------

def final_energy_gradient_dense(L: int, Jr: np.ndarray, h_steps, dt: float, h_target: float, psi0: np.ndarray):
    """Exact loss = <psi_N|H(h_target)|psi_N> with psi_k = expm(-i dt H(h_k)) psi_{k-1},
    H(h) = H_zz + h X, and its gradients with respect to every h_k and to the overall
    coupling scale s (J(r) -> s J(r) at s = 1, in the dynamics and in the target).

    dloss/dtheta = 2 Re sum_k <lambda_k| dU_k/dtheta |psi_{k-1}> (+ the target's own
    <psi_N|H_zz|psi_N> for s), lambda_N = H(h_target) psi_N, lambda_{k-1} = U_k^H lambda_k.
    dU_k/dtheta is the Frechet derivative of expm at A_k = -i dt H(h_k) in the
    direction E = dA_k/dtheta, read off the block-triangular exponential
    expm([[A, E], [0, A]]) = [[expm(A), L(A, E)], [0, expm(A)]] (Van Loan 1978).
    Dense: small L only.  Returns (loss, grad_h, grad_scale)."""
    Hzz = hamiltonian_dense(L, Jr, 0.0)
    X = hamiltonian_dense(L, np.zeros_like(Jr), 1.0)
    D = 1 << L
    hs = [float(x) for x in h_steps]
    U = [sla.expm(-1j * dt * (Hzz + hk * X)) for hk in hs]
    psis = [np.asarray(psi0, dtype=np.complex128)]
    for Uk in U:
        psis.append(Uk @ psis[-1])
    HT = Hzz + h_target * X
    psiN = psis[-1]
    loss = float(np.real(np.vdot(psiN, HT @ psiN)))
    lam = HT @ psiN
    grad_h = np.zeros(len(hs))
    gscale = float(np.real(np.vdot(psiN, Hzz @ psiN)))
    Z = np.zeros((D, D), dtype=np.complex128)
    for k in range(len(hs), 0, -1):
        A = -1j * dt * (Hzz + hs[k - 1] * X)
        for E, which in ((-1j * dt * X, "h"), (-1j * dt * Hzz, "s")):
            big = sla.expm(np.block([[A, E], [Z, A]]))
            Lk = big[:D, D:]
            val = 2.0 * float(np.real(np.vdot(lam, Lk @ psis[k - 1])))
            if which == "h":
                grad_h[k - 1] = val
            else:
                gscale += val
        lam = U[k - 1].conj().T @ lam
    return loss, grad_h, gscale


def final_energy_krylov(L: int, Jr: np.ndarray, h_steps, dt: float, m: int, h_target: float, psi0: np.ndarray,
                        scale: float = 1.0) -> float:
    """The same loss with every step taken by ``krylov_step`` (CSR products), couplings
    scaled by ``scale``: the forward model whose central differences give reference
    gradients beyond dense sizes."""
    Hzz = hamiltonian_csr(L, scale * np.asarray(Jr, dtype=np.float64), 0.0)
    X = hamiltonian_csr(L, np.zeros_like(np.asarray(Jr, dtype=np.float64)), 1.0)
    psi = np.asarray(psi0, dtype=np.complex128)
    for hk in h_steps:
        hk = float(hk)
        psi, _ = krylov_step(lambda v: Hzz @ v + hk * (X @ v), psi, dt, m)
    return float(np.real(np.vdot(psi, Hzz @ psi + h_target * (X @ psi))))


def exact_propagate_dense(H: np.ndarray, psi: np.ndarray, t: float) -> np.ndarray:
    """exp(-i H t) psi by the dense matrix exponential (method 1, Sec. III.A)."""
    return sla.expm(-1j * t * H) @ psi


# ---------------------------------------------------------------------------
# Measurements (Sec. IV)
# ---------------------------------------------------------------------------

def rdm_sites(psi: np.ndarray, L: int, sites) -> np.ndarray:
    """Reduced density matrix of the given sites (1-based), rho = A A^dagger.

    Reshape psi to a rank-L tensor, move the kept indices to the front, view
    as a (2^l, rest) matrix A and form A A^dagger (Sec. IV, single- and
    two-site reduced density matrices).
    """
    T = psi.reshape((2,) * L)
    keep = [s - 1 for s in sites]
    rest = [a for a in range(L) if a not in keep]
    A = np.transpose(T, keep + rest).reshape(1 << len(keep), -1)
    return A @ A.conj().T


def measure_local(psi: np.ndarray, L: int) -> np.ndarray:
    """<sz_k> = Tr(sz rho_k) for k = 1..L."""
    return np.array([float(np.real(np.trace(SZ @ rdm_sites(psi, L, [k])))) for k in range(1, L + 1)])


def measure_corr(psi: np.ndarray, L: int) -> np.ndarray:
    """<sz_i sz_j> = Tr((sz x sz) rho_ij) as an L x L matrix (diagonal = <psi|psi>)."""
    ZZ = np.kron(SZ, SZ)
    C = np.zeros((L, L))
    nrm2 = float(np.real(np.vdot(psi, psi)))
    for i in range(1, L + 1):
        C[i - 1, i - 1] = nrm2
        for j in range(i + 1, L + 1):
            v = float(np.real(np.trace(ZZ @ rdm_sites(psi, L, [i, j]))))
            C[i - 1, j - 1] = C[j - 1, i - 1] = v
    return C


def measure_corr_pair(psi: np.ndarray, L: int, i: int, j: int) -> float:
    """One correlator <sz_i sz_j> through the two-site reduced density matrix."""
    ZZ = np.kron(SZ, SZ)
    return float(np.real(np.trace(ZZ @ rdm_sites(psi, L, [i, j]))))


def schmidt_spectrum(psi: np.ndarray, L: int, cut: int | None = None) -> np.ndarray:
    """Eigenvalues of rho_l = M M^dagger, M = psi as a (2^l, 2^(L-l)) matrix.

    Sec. IV, bond entropy: left block = sites 1..l; l = floor(L/2) by default.
    Returned in descending order.
    """
    l = L // 2 if cut is None or cut < 0 else cut
    M = psi.reshape(1 << l, 1 << (L - l))
    rho = M @ M.conj().T
    return np.sort(np.linalg.eigvalsh(rho))[::-1]


def schmidt_spectrum_small(psi: np.ndarray, L: int, cut: int | None = None) -> np.ndarray:
    """The 2^min(l, L-l) Schmidt values of the cut after site l, descending.

    Sec. IV, bond entropy: rho_A = M M^dagger and rho_B = (M^dagger M)^T have the
    same nonzero spectrum (the squared singular values of M), so the smaller of
    the two Gram matrices is diagonalised.
    """
    l = L // 2 if cut is None or cut < 0 else cut
    M = psi.reshape(1 << l, 1 << (L - l))
    G = M @ M.conj().T if l <= L - l else M.conj().T @ M
    return np.sort(np.linalg.eigvalsh(G))[::-1]


def entropy_from_spectrum(lam: np.ndarray) -> float:
    """S = -sum_j Lambda_j ln Lambda_j (natural log); Lambda <= 0 counts as 0."""
    lam = np.asarray(lam, dtype=np.float64)
    pos = lam[lam > 0.0]
    return float(-np.sum(pos * np.log(pos)))


def schmidt_entropy(psi: np.ndarray, L: int, cut: int | None = None) -> float:
    return entropy_from_spectrum(schmidt_spectrum(psi, L, cut))


def energy(matvec, psi: np.ndarray) -> float:
    """<psi|H|psi> (energy measurement)."""
    return float(np.real(np.vdot(psi, matvec(psi))))


# ---------------------------------------------------------------------------
# Error measures and convergence rate (Sec. V, Eqs. erhoi-eentr, convrate)
# ---------------------------------------------------------------------------

def trace_distance(rho: np.ndarray, sigma: np.ndarray) -> float:
    """D = 1/2 |rho - sigma|_1 with |A| = sqrt(A^dagger A)."""
    ev = np.linalg.eigvalsh(rho - sigma)
    return 0.5 * float(np.sum(np.abs(ev)))


def eps_local(psi: np.ndarray, ref: np.ndarray, L: int) -> float:
    """Maximal single-site trace distance over all sites (Eq. erhoi)."""
    return max(trace_distance(rdm_sites(psi, L, [k]), rdm_sites(ref, L, [k])) for k in range(1, L + 1))


def convergence_rate(eps_big: float, eps_small: float, ratio: float) -> float:
    """r = ln(eps(ratio*dt)/eps(dt)) / ln(ratio) (Eq. convrate)."""
    return math.log(eps_big / eps_small) / math.log(ratio)
