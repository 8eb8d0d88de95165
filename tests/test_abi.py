"""The C-ABI library loads and exports every symbol include/osmps_ed.h declares
(CPU only: no call here touches a GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_symbols():
    names = set()
    for hdr in HEADERS:
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(osmps_ed_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("osmps_ed_create", "osmps_ed_apply_H", "osmps_ed_lanczos_ground", "osmps_ed_krylov_evolve",
                     "osmps_ed_measure_local", "osmps_ed_measure_corr", "osmps_ed_schmidt_entropy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1802_10052_gb300 as pkg
    so = C.CDLL(pkg.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(so, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1802_10052_gb300 import _binding
    assert set(_binding.SIGNATURES) == set(declared_symbols())


def test_strerror_and_host_side_argument_checks():
    from paper_1802_10052_gb300 import _binding as B
    lib = B.lib
    assert lib.osmps_ed_strerror(B.OSMPS_OK) == b"success"
    assert lib.osmps_ed_strerror(B.OSMPS_EINVAL) == b"invalid argument"
    h = C.c_void_p()
    # rejected before any CUDA call
    assert lib.osmps_ed_create(0, None, 1.0, 1.0, 1.0, 0, None, C.byref(h)) == B.OSMPS_EINVAL
    assert lib.osmps_ed_create(31, None, 1.0, 1.0, 1.0, 0, None, C.byref(h)) == B.OSMPS_EINVAL
    assert lib.osmps_ed_create(8, None, 1.0, 1.0, float("nan"), 0, None, C.byref(h)) == B.OSMPS_EINVAL
    assert lib.osmps_ed_create(8, None, 1.0, 1.0, 1.0, 7, None, C.byref(h)) == B.OSMPS_EINVAL
    assert lib.osmps_ed_create(8, None, 1.0, 1.0, 1.0, 0, None, None) == B.OSMPS_EINVAL
    bad = (C.c_double * 7)(*([1.0] * 6 + [float("inf")]))
    assert lib.osmps_ed_create(8, bad, 1.0, 1.0, 1.0, 0, None, C.byref(h)) == B.OSMPS_EINVAL
    assert lib.osmps_ed_destroy(None) == B.OSMPS_OK
    assert lib.osmps_ed_apply_H(None, None, None) == B.OSMPS_EINVAL
    assert lib.osmps_ed_krylov_evolve(None, None, 0.1, 1, 20, 0.0, None) == B.OSMPS_EINVAL
    # scheduling entry points: a null handle is rejected before any CUDA call
    S = C.c_double()
    assert lib.osmps_ed_schmidt_entropy_async(None, None, -1, C.byref(S), None) == B.OSMPS_EINVAL
    assert lib.osmps_ed_measure_wait(None) == B.OSMPS_EINVAL
    assert lib.osmps_ed_set_async_eigensolver(None, 16) == B.OSMPS_EINVAL
    assert lib.osmps_ed_set_sm_count(None, 8) == B.OSMPS_EINVAL
    assert lib.osmps_ed_set_prefetch(None, 1) == B.OSMPS_EINVAL


def test_batch_host_side_argument_checks():
    """osmps_ed_batch_create rejects bad arguments before touching CUDA."""
    from paper_1802_10052_gb300 import _binding as B
    lib = B.lib
    h = C.c_void_p()

    def create(Ls, prec=B.OSMPS_MIXED, max_iter=100, hval=1.0, out=True):
        n = len(Ls)
        La = (C.c_int * max(n, 1))(*Ls)
        one = (C.c_double * max(n, 1))(*([1.0] * max(n, 1)))
        hh = (C.c_double * max(n, 1))(*([hval] * max(n, 1)))
        return lib.osmps_ed_batch_create(n, La, one, one, hh, prec, max_iter, None, C.byref(h) if out else None)

    assert create([14], out=False) == B.OSMPS_EINVAL
    assert create([]) == B.OSMPS_EINVAL
    assert create([0]) == B.OSMPS_EINVAL
    assert create([31]) == B.OSMPS_EINVAL
    assert create([14], prec=5) == B.OSMPS_EINVAL
    assert create([14], max_iter=0) == B.OSMPS_EINVAL
    assert create([14], max_iter=1001) == B.OSMPS_EINVAL
    assert create([14], hval=float("nan")) == B.OSMPS_EINVAL
    # valid chains outside the tile range of the batched solver
    assert create([12]) == B.OSMPS_EUNSUPPORTED
    assert create([11], prec=B.OSMPS_FP64) == B.OSMPS_EUNSUPPORTED
    assert create([14, 23]) == B.OSMPS_EUNSUPPORTED
    assert lib.osmps_ed_batch_destroy(None) == B.OSMPS_EINVAL
    assert lib.osmps_ed_batch_lanczos_ground(None, None, 1e-10, None, None, None, None) == B.OSMPS_EINVAL
    assert lib.osmps_ed_batch_check(None) == B.OSMPS_EINVAL
