"""Adjoint gradients of a final energy under a piecewise-constant field through
the C ABI: against the oracle's exact (block-exponential) gradient, against
oracle central differences of its Krylov forward model, and at the full
L = 20, 200-step size against central differences (step 1e-6, FP64)."""
import time

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


@pytest.mark.parametrize("prec,L,tol", [("fp64", 6, 1e-10), ("fp64", 8, 1e-10), ("mixed", 8, 1e-5), ("mixed", 10, 1e-5)])
def test_adjoint_matches_exact_gradient(prec, L, tol):
    hs = si.field_schedule(12, seed=4)
    dt = 0.05
    Jr = O.coupling_table(L, 1.0, 2.0)
    psi0 = si.basis_state(L, 0)
    loss_o, gh_o, gs_o = O.final_energy_gradient_dense(L, Jr, hs, dt, 1.0, psi0)
    c = Chain(L, J=1.0, alpha=2.0, h=1.0, prec=prec)
    x = to_dev(psi0, prec)
    loss, gh, gs = c.adjoint_grad(x, hs, dt, m=24, h_target=1.0, stride=4, nquad=8)
    scale = max(1.0, np.max(np.abs(gh_o)), abs(gs_o))
    assert abs(loss - loss_o) <= tol * max(1.0, abs(loss_o))
    assert np.max(np.abs(gh - gh_o)) <= tol * scale, np.max(np.abs(gh - gh_o))
    assert abs(gs - gs_o) <= tol * scale
    # psi0 untouched
    np.testing.assert_array_equal(x.cpu().numpy(), psi0.astype(x.cpu().numpy().dtype))


def test_adjoint_stride_and_quadrature_independence():
    L, hs, dt = 8, si.field_schedule(10, seed=9), 0.04
    c = Chain(L, J=1.0, alpha=2.0, h=1.0, prec="fp64")
    x = to_dev(si.basis_state(L, 0), "fp64")
    ref = c.adjoint_grad(x, hs, dt, m=24, stride=1, nquad=10)
    for stride, nq in ((3, 8), (10, 12)):
        out = c.adjoint_grad(x, hs, dt, m=24, stride=stride, nquad=nq)
        assert abs(out[0] - ref[0]) < 1e-12 * abs(ref[0])
        assert np.max(np.abs(out[1] - ref[1])) < 1e-10 * np.max(np.abs(ref[1]))
        assert abs(out[2] - ref[2]) < 1e-10 * abs(ref[2])


def test_adjoint_against_oracle_differences_L12():
    """L = 12, 200 steps: gradients against central differences of the oracle's own
    Krylov forward model (CSR products, FP64) for sampled steps and the scale."""
    L, n, dt, m = 12, 200, 0.025, 20
    hs = si.field_schedule(n, seed=4)
    Jr = O.coupling_table(L, 1.0, 2.0)
    psi0 = si.basis_state(L, 0)
    c = Chain(L, J=1.0, alpha=2.0, h=1.0, prec="fp64")
    loss, gh, gs = c.adjoint_grad(to_dev(psi0, "fp64"), hs, dt, m=m, h_target=1.0)
    assert abs(loss - O.final_energy_krylov(L, Jr, hs, dt, m, 1.0, psi0)) < 1e-10 * abs(loss)
    eps = 1e-6
    for k in (0, 117, 199):
        hp, hm = hs.copy(), hs.copy()
        hp[k] += eps
        hm[k] -= eps
        fd = (O.final_energy_krylov(L, Jr, hp, dt, m, 1.0, psi0) - O.final_energy_krylov(L, Jr, hm, dt, m, 1.0, psi0)) / (2 * eps)
        assert abs(gh[k] - fd) < 1e-6 * max(1.0, np.max(np.abs(gh))), (k, gh[k], fd)
    fd = (O.final_energy_krylov(L, Jr, hs, dt, m, 1.0, psi0, scale=1 + eps)
          - O.final_energy_krylov(L, Jr, hs, dt, m, 1.0, psi0, scale=1 - eps)) / (2 * eps)
    assert abs(gs - fd) < 1e-6 * max(1.0, abs(gs))


def test_adjoint_full_size_L20():
    """L = 20, alpha = 2, 200 steps of dt = 0.025 with h_k ~ U[0.5, 1.5] (seed 4), from
    all up, loss = <H(h = 1)>: every gradient against central differences (step 1e-6,
    FP64) of the same forward model for sampled steps and the coupling scale, and the
    autograd wrapper's gradients equal to the direct call's."""
    from paper_1802_10052_gb300 import FinalEnergy

    L, n, dt, m = 20, 200, 0.025, 20
    hs = si.field_schedule(n, seed=4)
    c = Chain(L, J=1.0, alpha=2.0, h=1.0, prec="fp64")
    x = c.new_state()
    c.init_basis_state(x, 0)
    t0 = time.perf_counter()
    loss, gh, gs = c.adjoint_grad(x, hs, dt, m=m, h_target=1.0)
    print(f"L=20 adjoint gradient: {time.perf_counter() - t0:.2f} s")
    eps = 1e-6

    def fwd(h, chain=c):
        return chain.adjoint_grad(x, h, dt, m=m, h_target=1.0, want_grad=False)[0]

    for k in (3, 101, 199):
        hp, hm = hs.copy(), hs.copy()
        hp[k] += eps
        hm[k] -= eps
        fd = (fwd(hp) - fwd(hm)) / (2 * eps)
        assert abs(gh[k] - fd) < 1e-6 * max(1.0, np.max(np.abs(gh))), (k, gh[k], fd)
    Jp = [(1 + eps) / r ** 2 for r in range(1, L)]
    Jm = [(1 - eps) / r ** 2 for r in range(1, L)]
    cp = Chain(L, couplings=Jp, h=1.0, prec="fp64")
    cm = Chain(L, couplings=Jm, h=1.0, prec="fp64")
    fd = (fwd(hs, cp) - fwd(hs, cm)) / (2 * eps)
    assert abs(gs - fd) < 1e-6 * max(1.0, abs(gs))
    h_t = torch.tensor(hs, dtype=torch.float64, requires_grad=True)
    s_t = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    out = FinalEnergy.apply(h_t, s_t, c, x, dt, m, 1.0)
    out.backward()
    assert abs(out.item() - loss) < 1e-12 * abs(loss)
    np.testing.assert_allclose(h_t.grad.numpy(), gh, rtol=0, atol=1e-12 * np.max(np.abs(gh)))
    assert abs(float(s_t.grad) - gs) < 1e-12 * abs(gs)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_adjoint_kept_bases_are_bit_identical(prec):
    """With checkpoints every step (stride 1) every backward step rebuilds the Krylov
    basis of psi_{k-1}; with stride 4 the bases built while recomputing a segment are
    kept and reused.  Same kernels on the same inputs in the same order: the loss
    and every gradient agree bit for bit."""
    L, hs, dt = 10, si.field_schedule(16, seed=11), 0.03
    c = Chain(L, J=1.0, alpha=2.0, h=1.0, prec=prec)
    x = to_dev(si.basis_state(L, 0), prec)
    a = c.adjoint_grad(x, hs, dt, m=16, stride=1, nquad=8)
    b = c.adjoint_grad(x, hs, dt, m=16, stride=4, nquad=8)
    assert a[0] == b[0] and a[2] == b[2]
    np.testing.assert_array_equal(a[1], b[1])
    c.close()
