"""The allocation-free measurement entry point against the handle-based one.

osmps_ed_measure_zz_noalloc serves callers that must not allocate device
memory at run time -- their device memory belongs to another allocator or
budget (a framework's caching pool), or they cannot afford the device-wide
synchronisation of cudaMalloc/cudaFree.  It works from a fixed scratch array
inside the library, shared by all calls.  Two calls in a row must agree with
osmps_ed_measure_zz (which uses the handle's own scratch) within the
tolerances of the other measurement tests.
"""
import ctypes as C
import math

import numpy as np
import pytest
import torch

import seeded_inputs as si

pytestmark = pytest.mark.gpu


def _noalloc(B, L, prec, psi, out):
    return B.lib.osmps_ed_measure_zz_noalloc(L, B.OSMPS_FP64 if prec == "fp64" else B.OSMPS_MIXED,
                                             C.c_void_p(psi.data_ptr()), C.c_void_p(out.data_ptr()),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_handle_entry_point(prec):
    from paper_1802_10052_gb300 import Chain
    from paper_1802_10052_gb300 import _binding as B
    tol = 1e-13 if prec == "fp64" else 1e-6
    dt = np.complex128 if prec == "fp64" else np.complex64
    for L, seed in [(14, 1), (22, 2)]:
        c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec=prec)
        psi = torch.from_numpy(si.gaussian_state(L, seed).astype(dt)).cuda()
        sz, zz = c.measure_zz(psi)
        out = torch.empty(L + L * L, dtype=torch.float64, device="cuda")
        for _ in range(2):  # two calls in a row share the library's scratch
            out.fill_(float("nan"))
            assert _noalloc(B, L, prec, psi, out) == B.OSMPS_OK
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_allclose(got[:L], sz, rtol=0, atol=tol)
            np.testing.assert_allclose(got[L:].reshape(L, L), zz, rtol=0, atol=tol)
        c.close()


def test_noalloc_rejects_sizes_beyond_the_maximum():
    from paper_1802_10052_gb300 import _binding as B
    psi = torch.zeros(4, dtype=torch.complex128, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert _noalloc(B, 31, "fp64", psi, out) == B.OSMPS_EINVAL
    assert _noalloc(B, 0, "fp64", psi, out) == B.OSMPS_EINVAL


@pytest.mark.timeout(600)
def test_noalloc_full_size_product_state_closed_form():
    """L = 28 complex64 (683 tiles per CTA of the 96-CTA pass): the rotated product
    state prod_k (cos q |up> - i sin q |down>) has <sz_k> = cos 2q and
    <sz_i sz_j> = cos^2 2q exactly; both entry points meet that within the mixed
    tolerance, low-bit sites included (their marginal is summed over every tile
    a CTA visits)."""
    from paper_1802_10052_gb300 import Chain
    from paper_1802_10052_gb300 import _binding as B
    L, q = 28, 0.3
    one = torch.tensor([math.cos(q), -1j * math.sin(q)], dtype=torch.complex64, device="cuda")
    psi = one
    for _ in range(L - 1):
        psi = torch.kron(psi, one)
    want_z, want_zz = math.cos(2 * q), math.cos(2 * q) ** 2
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="mixed")
    sz, zz = c.measure_zz(psi)
    off = ~np.eye(L, dtype=bool)
    np.testing.assert_allclose(sz, want_z, rtol=0, atol=1e-5)
    np.testing.assert_allclose(zz[off], want_zz, rtol=0, atol=1e-5)
    out = torch.empty(L + L * L, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        assert _noalloc(B, L, "mixed", psi, out) == B.OSMPS_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[:L], want_z, rtol=0, atol=1e-5)
        np.testing.assert_allclose(got[L:].reshape(L, L)[off], want_zz, rtol=0, atol=1e-5)
        np.testing.assert_allclose(got[L:].reshape(L, L), zz, rtol=0, atol=1e-6)
    c.close()
