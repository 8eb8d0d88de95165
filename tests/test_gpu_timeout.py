"""Failure path of the bounded device waits, made to run out on purpose in the
allowed form: a kernel waits on an mbarrier phase that nothing completes, with
the same bounded wait the H.psi and Gram kernels use and a short limit.  No
fault, trap or hang: the wait gives up, raises the handle's error word, the
next synchronising call returns OSMPS_ETIMEOUT, and the handle keeps working."""
import ctypes as C

import numpy as np
import pytest
import torch

import seeded_inputs as si
from oracle import ed_oracle as O
from _gpu import to_dev

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_handle_recovers():
    from paper_1802_10052_gb300 import Chain
    from paper_1802_10052_gb300 import _binding as B
    L = 12
    c = Chain(L, J=1.0, alpha=1.5, h=0.8, prec="fp64")
    x = to_dev(si.gaussian_state(L, 21), "fp64")
    want = O.energy(O.RuleSetH(L, O.coupling_table(L, 1.0, 1.5), 0.8), x.cpu().numpy())
    e, n2 = C.c_double(), C.c_double()
    # a wait that nothing completes gives up after 50 ms
    assert B.lib.osmps_ed_probe_wait(c._h, 0.05, 0) == B.OSMPS_OK
    assert B.lib.osmps_ed_energy(c._h, C.c_void_p(x.data_ptr()), C.byref(e), C.byref(n2)) == B.OSMPS_ETIMEOUT
    # the error word was cleared by that report: the handle computes again
    assert B.lib.osmps_ed_energy(c._h, C.c_void_p(x.data_ptr()), C.byref(e), C.byref(n2)) == B.OSMPS_OK
    assert abs(e.value - want) < 1e-10 * abs(want)
    y = c.new_state()
    c.apply_H(x, y)
    ref = O.RuleSetH(L, O.coupling_table(L, 1.0, 1.5), 0.8)(x.cpu().numpy())
    assert np.linalg.norm(y.cpu().numpy() - ref) < 1e-10 * np.linalg.norm(ref)
    # a wait whose phase completes reports nothing
    assert B.lib.osmps_ed_probe_wait(c._h, 0.05, 1) == B.OSMPS_OK
    assert B.lib.osmps_ed_energy(c._h, C.c_void_p(x.data_ptr()), C.byref(e), C.byref(n2)) == B.OSMPS_OK
    # out-of-range limits are argument errors, never a longer wait
    assert B.lib.osmps_ed_probe_wait(c._h, 0.0, 0) == B.OSMPS_EINVAL
    assert B.lib.osmps_ed_probe_wait(c._h, 2.5, 0) == B.OSMPS_EINVAL
    c.close()
    torch.cuda.synchronize()
