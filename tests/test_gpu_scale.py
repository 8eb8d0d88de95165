"""The scale workload (H_LRQI at L = 30, alpha = 1, h = 1.2, complex64, Krylov
dimension 12, quench from the Neel state at dt = 0.02) at full size: the oracle
cannot hold this state, so the checks are properties that hold at any size,
plus the sampled-row H.psi parity in test_gpu_hpsi.py."""
import numpy as np
import pytest
import torch

import seeded_inputs as si

pytestmark = pytest.mark.gpu

L, ALPHA, H = 30, 1.0, 1.2


def Chain(*a, **k):
    from paper_1802_10052_gb300 import Chain as _C
    return _C(*a, **k)


def neel_energy():
    # the Neel state is an eigenstate of the diagonal part: sum_r (L - r) (-1)^r / r^alpha
    return sum((L - r) * (-1) ** r / r ** ALPHA for r in range(1, L))


@pytest.mark.timeout(900)
def test_scale_L30_neel_quench_and_half_chain_spectrum():
    c = Chain(L, J=1.0, alpha=ALPHA, h=H, prec="mixed")
    x = c.new_state()
    c.init_basis_state(x, si.neel_index(L))
    e0, n0 = c.energy(x)
    assert abs(n0 - 1.0) < 1e-6
    assert abs(e0 - neel_energy()) < 1e-5 * abs(e0)
    y = x.clone()
    c.krylov_evolve(x, 0.02, 1, 12)
    c.krylov_evolve(y, 0.01, 2, 12)
    e1, n1 = c.energy(x)
    assert abs(n1 - 1.0) < 1e-5                    # unitary
    assert abs(e1 - e0) < 1e-5 * abs(e0)           # energy conserved
    # one step of 0.02 and two of 0.01 give the same state (converged Krylov steps)
    assert torch.linalg.vector_norm(x - y).item() < 5e-5
    del y
    # reflection times global spin flip maps the Neel state to itself and commutes with H
    sz = c.measure_local(x)
    np.testing.assert_allclose(sz, -sz[::-1], atol=1e-5)
    assert np.all(np.abs(np.abs(sz) - 1.0) < 0.05) and sz[0] > 0   # still close to the Neel pattern
    c.close()
    torch.cuda.empty_cache()
    # half-chain spectrum through the tensor-core Gram product, 32768 x 32768
    m = Chain(L, J=1.0, alpha=ALPHA, h=H, prec="mixed")
    S, lam = m.schmidt_entropy(x, spectrum=True)
    assert len(lam) == 1 << 15
    assert np.all(np.isfinite(lam))
    assert abs(lam.sum() - 1.0) < 1e-4
    assert 0.99 < lam[0] <= 1.0 + 1e-5              # close to a product state after t = 0.02
    assert np.all(np.diff(lam) <= 0.0)
    assert 0.0 <= S < 0.1
    m.close()


@pytest.mark.timeout(1500)
def test_scale_L30_full_quench_to_t2():
    """The whole scale workload: 100 Krylov steps of 0.02 (m = 12) from the Neel
    state to t = 2.  Every step: unitarity and energy conservation within the
    mixed tolerance.  At t = 2: the reflection x spin-flip symmetry of <sz_i>.
    Beside it the same quench at L = 28 in complex64 against the FP64 form
    (whose layout is checked against the oracle at L = 24): <sz_i>, <sz_i sz_j>
    and the state within the mixed tolerance after all 100 steps."""
    c = Chain(L, J=1.0, alpha=ALPHA, h=H, prec="mixed")
    x = c.new_state()
    c.init_basis_state(x, si.neel_index(L))
    e0 = neel_energy()
    for k in range(100):
        c.krylov_evolve(x, 0.02, 1, 12)
        e, n2 = c.energy(x)
        assert abs(n2 - 1.0) < 1e-5, (k, n2)
        assert abs(e / n2 - e0) < 1e-5 * abs(e0), (k, e, e0)
    sz = c.measure_local(x)
    np.testing.assert_allclose(sz, -sz[::-1], atol=1e-5)
    c.close()
    del x
    torch.cuda.empty_cache()
    L28 = 28
    out = {}
    for prec in ("fp64", "mixed"):
        m = Chain(L28, J=1.0, alpha=ALPHA, h=H, prec=prec)
        y = m.new_state()
        m.init_basis_state(y, si.neel_index(L28))
        m.krylov_evolve(y, 0.02, 100, 12)
        sz28, zz28 = m.measure_zz(y)
        out[prec] = (y.to(torch.complex128), sz28, zz28)
        m.close()
        del y
        torch.cuda.empty_cache()
    yf, szf, zzf = out["fp64"]
    ym, szm, zzm = out["mixed"]
    np.testing.assert_allclose(szm, szf, rtol=0, atol=1e-5)
    np.testing.assert_allclose(zzm, zzf, rtol=0, atol=1e-5)
    assert (torch.linalg.vector_norm(ym - yf) / torch.linalg.vector_norm(yf)).item() < 1e-5
