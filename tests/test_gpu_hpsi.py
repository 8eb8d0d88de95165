"""H.psi through the C ABI against the FP64 oracle (element by element)."""
import numpy as np
import pytest
import torch

import seeded_inputs as si
from oracle import ed_oracle as O
from _gpu import TOL, Gathered, rel, seeded_device_state, to_dev, to_host

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "mixed"]


def chain_for(L, Jr, hk, prec):
    from paper_1802_10052_gb300 import Chain
    c = Chain(L, couplings=list(Jr), prec=prec)
    c.set_site_fields(list(hk))
    return c


@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 7, 8, 11, 12, 13, 14, 15, 16, 17, 18, 20])
def test_apply_H_matches_csr(L, prec, threads):
    """Both CTA shapes of the passes (16 or 8 vectors per thread)."""
    rng = np.random.default_rng(100 + L)
    Jr = rng.normal(size=L - 1)
    hk = rng.normal(size=L)
    c = chain_for(L, Jr, hk, prec)
    c.set_pass_threads(threads)
    psi = si.gaussian_state(L, L)
    x = to_dev(psi, prec)
    ref = O.hamiltonian_csr(L, Jr, hk) @ x.cpu().numpy().astype(np.complex128)
    out = c.new_state()
    c.apply_H(x, out)
    got = to_host(out)
    tol = 1e-13 if prec == "fp64" else 1e-6
    scale = np.max(np.abs(ref))
    np.testing.assert_allclose(got, ref, rtol=0, atol=tol * scale * 10)
    assert rel(got, ref) < tol


@pytest.mark.parametrize("prec", PRECS)
def test_apply_H_models_and_signs(prec):
    # nearest neighbour (alpha=None) and power law, both signs, uniform field
    from paper_1802_10052_gb300 import Chain
    L = 15
    psi = si.gaussian_state(L, 3)
    for J, alpha, h in [(-1.0, None, -1.0), (1.0, 1.5, 0.8), (-0.7, 0.0, 2.0), (1.0, 3.0, -0.3)]:
        c = Chain(L, J=J, alpha=alpha, h=h, prec=prec)
        Jr = O.coupling_table(L, J, alpha)
        x = to_dev(psi, prec)
        ref = O.RuleSetH(L, Jr, h)(x.cpu().numpy().astype(np.complex128))
        out = c.new_state()
        c.apply_H(x, out)
        assert rel(to_host(out), ref) < (1e-13 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("prec", PRECS)
def test_apply_H_product_states_and_set_field(prec):
    from paper_1802_10052_gb300 import Chain
    L = 16
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec=prec)
    x = c.new_state()
    Jr = O.coupling_table(L, 1.0, 1.5)
    for b in (0, si.neel_index(L), (1 << L) - 1, 12345):
        c.init_basis_state(x, b)
        out = c.new_state()
        c.apply_H(x, out)
        got = to_host(out)
        ref = O.apply_H_rows(L, Jr, 0.8, si.basis_state(L, b), np.arange(1 << L))
        assert rel(got, ref) < (1e-14 if prec == "fp64" else 1e-7)
    c.set_field(0.0)
    c.init_basis_state(x, 777)
    c.apply_H(x, out)
    got = to_host(out)
    E = O.diagonal_energy(L, Jr, np.array([777]))[0]
    assert abs(got[777] - E) < 1e-12 * abs(E) + (1e-5 if prec == "mixed" else 0)
    assert np.count_nonzero(got) == 1


def test_energy_call():
    from paper_1802_10052_gb300 import Chain
    L = 14
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="fp64")
    psi = si.gaussian_state(L, 5) * 1.7
    x = to_dev(psi, "fp64")
    e, n2 = c.energy(x)
    ref = O.RuleSetH(L, O.coupling_table(L, 1.0, 1.5), 0.8)
    assert abs(e - np.vdot(psi, ref(psi)).real) < 1e-12 * abs(e)
    assert abs(n2 - np.vdot(psi, psi).real) < 1e-13


@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("L,prec", [(24, "fp64"), (24, "mixed"), (28, "mixed"), (28, "fp64"), (30, "mixed")])
def test_apply_H_full_size_sampled_rows(L, prec, threads):
    """At the workload sizes: rows sampled across the whole index range, each
    checked against the oracle's row-definition product (both CTA shapes)."""
    from paper_1802_10052_gb300 import Chain
    alpha, h = (1.5, 0.8) if L != 30 else (1.0, 1.2)
    c = Chain(L, J=1.0, alpha=alpha, h=h, prec=prec)
    c.set_pass_threads(threads)
    x = seeded_device_state(L, 28, prec)
    out = c.new_state()
    c.apply_H(x, out)
    torch.cuda.synchronize()
    rng = np.random.default_rng(L)
    rows = np.concatenate([rng.integers(0, 1 << L, size=3000), [0, 1, (1 << L) - 1, (1 << (L - 1)), 8191, 8192]])
    Jr = O.coupling_table(L, 1.0, alpha)
    ref = O.apply_H_rows(L, Jr, h, Gathered(x), rows)
    got = Gathered(out)[rows]
    assert rel(got, ref) < (1e-13 if prec == "fp64" else 1e-6)
    del out, x, c
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("L", [13, 20, 24])
def test_prefetch_and_sm_count_do_not_change_the_product(L, prec):
    """The L2 prefetch distance and the grid size schedule memory traffic only:
    H.psi is bit-identical across them (no reduction enters the output)."""
    c = chain_for(L, [1.0 / r ** 1.5 for r in range(1, L)], [0.8] * L, prec)
    x = to_dev(si.gaussian_state(L, 3 * L), prec)
    ref = c.new_state()
    c.set_prefetch(0)
    c.apply_H(x, ref)
    out = c.new_state()
    for pf, nsm in ((1, 0), (2, 0), (3, 0), (1, 96), (0, 17)):
        c.set_prefetch(pf)
        c.set_sm_count(nsm)
        c.apply_H(x, out)
        assert torch.equal(out, ref), (pf, nsm)
    c.close()


@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("L", [3, 8, 12, 13, 14, 18, 20])
@pytest.mark.parametrize("mode", [0, 1, 7])
def test_fp64_flip_sums_match_csr(L, mode, threads):
    """complex128 H.psi with the flip sums in 64-bit fixed point (mode 1: every pass whose
    flipped bits share one field; mode 7: only passes of seven or more flipped bits) and on
    FP64 multiply-adds (mode 0), uniform and site-dependent fields, against the CSR product."""
    from paper_1802_10052_gb300 import Chain
    rng = np.random.default_rng(500 + L)
    Jr = rng.normal(size=L - 1)
    psi = si.gaussian_state(L, 7 + L)
    x = to_dev(psi, "fp64")
    for hk in ([0.83] * L, list(rng.normal(size=L))):
        c = chain_for(L, Jr, hk, "fp64")
        c.set_flip_sums(mode)
        c.set_pass_threads(threads)
        out = c.new_state()
        c.apply_H(x, out)
        ref = O.hamiltonian_csr(L, Jr, hk) @ psi
        got = to_host(out)
        assert rel(got, ref) < 1e-13
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)) * 10)
        c.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_fp64_flip_sums_wide_dynamic_range(mode):
    """Amplitudes spread over sixty decades (1e-30 .. 1).  FP64 multiply-adds (mode 0):
    every output element, small ones included, to 1e-12 of its own size plus 1e-30 of the
    largest.  Fixed-point sums (mode 1): each flip sum is exact up to one unit of 2^-57 of
    its tile's largest amplitude per flipped partner (at most 12 of them), so an element may
    also be off by 12 * 2^-57 h max|psi| plus the rounding of the sum; the whole product
    stays within the FP64 tolerance."""
    L = 14
    rng = np.random.default_rng(77)
    psi = si.gaussian_state(L, 77) * 10.0 ** rng.uniform(-30, 0, size=1 << L)
    Jr = O.coupling_table(L, 1.0, 1.5)
    ref = O.RuleSetH(L, Jr, 0.8)(psi)
    from paper_1802_10052_gb300 import Chain
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="fp64")
    c.set_flip_sums(mode)
    x = to_dev(psi, "fp64")
    out = c.new_state()
    c.apply_H(x, out)
    got = to_host(out)
    bound = np.abs(O.RuleSetH(L, np.abs(Jr), 0.8)(np.abs(psi))) + np.abs(O.diagonal_energy(L, Jr, np.arange(1 << L)) * psi)
    mx = np.max(np.abs(psi))
    fixed = 0.0 if mode == 0 else 0.8 * 12 * 2.0 ** -57 * mx
    assert np.all(np.abs(got - ref) <= 1e-12 * bound + fixed + 1e-30 * mx)
    assert rel(got, ref) < 1e-13
    c.close()
