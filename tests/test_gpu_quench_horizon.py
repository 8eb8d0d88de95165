"""The long-range quench workload over its whole horizon: H = sum |i-j|^-1.5 sz sz
+ 0.8 sum sx, L = 24, all-up start, Krylov m = 20, dt = 0.01 to t = 5, with
<sz_i>, <sz_i sz_j> and the half-chain entropy at t = 0, 0.1, ..., 5 (51 points).
The complex64 form against the FP64 form at every point within the mixed
tolerance (Sec. V error measures: local observables, correlators, entropy),
and the FP64 form against what exact evolution conserves (norm, and the energy
sum_r (L - r) J(r) of the all-up state).  The FP64 form's parity with the
oracle at this size is in test_gpu_lanczos_krylov.py."""
import numpy as np
import pytest
import torch

from _gpu import TOL

pytestmark = pytest.mark.gpu

L, ALPHA, H, M, DT = 24, 1.5, 0.8, 20, 0.01


def Chain(*a, **k):
    from paper_1802_10052_gb300 import Chain as _C
    return _C(*a, **k)


def trajectory(prec):
    c = Chain(L, J=1.0, alpha=ALPHA, h=H, prec=prec)
    x = c.new_state()
    c.init_basis_state(x, 0)
    out = []
    for k in range(51):
        if k > 0:
            c.krylov_evolve(x, DT, 10, M)
        sz, zz = c.measure_zz(x)
        out.append((sz, zz, c.schmidt_entropy(x)))
    e, n2 = c.energy(x)
    c.close()
    del x
    torch.cuda.empty_cache()
    return out, e, n2


@pytest.mark.timeout(1800)
def test_quench_L24_full_horizon_mixed_against_fp64():
    ref, e64, n64 = trajectory("fp64")
    got, e32, n32 = trajectory("mixed")
    e0 = sum((L - r) / r ** ALPHA for r in range(1, L))
    assert abs(n64 - 1.0) < TOL["fp64"] and abs(e64 / n64 - e0) < TOL["fp64"] * abs(e0)
    assert abs(n32 - 1.0) < TOL["mixed"] and abs(e32 / n32 - e0) < TOL["mixed"] * abs(e0)
    for k, ((sz, zz, S), (sz0, zz0, S0)) in enumerate(zip(got, ref)):
        np.testing.assert_allclose(sz, sz0, rtol=0, atol=TOL["mixed"], err_msg=f"t={0.1 * k:.1f}")
        np.testing.assert_allclose(zz, zz0, rtol=0, atol=TOL["mixed"], err_msg=f"t={0.1 * k:.1f}")
        assert abs(S - S0) < TOL["mixed"], (0.1 * k, S, S0)
    # a product state at t = 0 (S = 0, every <sz_i> = 1) that the quench entangles
    assert ref[0][2] < 1e-12 and np.all(np.abs(ref[0][0] - 1.0) < 1e-12)
    assert ref[-1][2] > 1e-3
