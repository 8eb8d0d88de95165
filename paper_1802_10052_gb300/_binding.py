"""ctypes binding of libosmps_ed (include/osmps_ed.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the shared library.  There is no fallback: if the library is
missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libosmps_ed.so")

OSMPS_OK, OSMPS_EINVAL, OSMPS_ENOMEM, OSMPS_ECUDA, OSMPS_ENOCONV, OSMPS_ETIMEOUT, OSMPS_EUNSUPPORTED = range(7)
OSMPS_FP64, OSMPS_MIXED = 0, 1

_P = C.c_void_p
_D = C.c_double
_DP = C.POINTER(C.c_double)
_I = C.c_int
_U64 = C.c_uint64

# name -> (restype, argtypes); kept in the order of the header
SIGNATURES = {
    "osmps_ed_create": (_I, [_I, _DP, _D, _D, _D, _I, _P, C.POINTER(_P)]),
    "osmps_ed_destroy": (_I, [_P]),
    "osmps_ed_set_stream": (_I, [_P, _P]),
    "osmps_ed_set_field": (_I, [_P, _D]),
    "osmps_ed_set_site_fields": (_I, [_P, _DP]),
    "osmps_ed_set_reorth": (_I, [_P, _I]),
    "osmps_ed_set_gram_mode": (_I, [_P, _I]),
    "osmps_ed_dim": (_I, [_P, C.POINTER(_U64)]),
    "osmps_ed_device_bytes": (_I, [_P, C.POINTER(_U64)]),
    "osmps_ed_init_basis_state": (_I, [_P, _P, _U64]),
    "osmps_ed_upload": (_I, [_P, _P, _P]),
    "osmps_ed_download": (_I, [_P, _P, _P]),
    "osmps_ed_apply_H": (_I, [_P, _P, _P]),
    "osmps_ed_energy": (_I, [_P, _P, _DP, _DP]),
    "osmps_ed_lanczos_ground": (_I, [_P, _P, _D, _I, _DP, _DP, C.POINTER(_I)]),
    "osmps_ed_krylov_evolve": (_I, [_P, _P, _D, _I, _I, _D, _DP]),
    "osmps_ed_adjoint_grad": (_I, [_P, _P, _I, _D, _DP, _I, _D, _I, _I, _DP, _DP, _DP]),
    "osmps_ed_apply_gates": (_I, [_P, _P, _I, C.POINTER(_I), _DP]),
    "osmps_ed_trotter_evolve": (_I, [_P, _P, _D, _I, _I]),
    "osmps_ed_rdm_pairs": (_I, [_P, _P, _DP, _DP]),
    "osmps_ed_entropy_sweep": (_I, [_P, _P, _DP]),
    "osmps_ed_measure_local": (_I, [_P, _P, _DP]),
    "osmps_ed_measure_corr": (_I, [_P, _P, _DP]),
    "osmps_ed_measure_zz": (_I, [_P, _P, _DP, _DP]),
    "osmps_ed_measure_zz_noalloc": (_I, [_I, _I, _P, _P, _P]),
    "osmps_ed_schmidt_entropy": (_I, [_P, _P, _I, _DP, _DP]),
    "osmps_ed_schmidt_entropy_async": (_I, [_P, _P, _I, _DP, _DP]),
    "osmps_ed_measure_wait": (_I, [_P]),
    "osmps_ed_set_sm_count": (_I, [_P, _I]),
    "osmps_ed_set_async_eigensolver": (_I, [_P, _I]),
    "osmps_ed_set_prefetch": (_I, [_P, _I]),
    "osmps_ed_set_flip_sums": (_I, [_P, _I]),
    "osmps_ed_set_pass_threads": (_I, [_P, _I]),
    "osmps_ed_set_lanczos_fold": (_I, [_P, _I]),
    "osmps_ed_set_entropy_method": (_I, [_P, _I]),
    "osmps_ed_launch_count": (_I, [_P, C.POINTER(C.c_int64)]),
    "osmps_ed_probe_wait": (_I, [_P, _D, _I]),
    "osmps_ed_timing_enable": (_I, [_P, _I]),
    "osmps_ed_timing_read": (_I, [_P, _DP, C.POINTER(C.c_int64), _I]),
    "osmps_ed_batch_create": (_I, [_I, C.POINTER(_I), _DP, _DP, _DP, _I, _I, _P, C.POINTER(_P)]),
    "osmps_ed_batch_destroy": (_I, [_P]),
    "osmps_ed_batch_offsets": (_I, [_P, C.POINTER(_U64)]),
    "osmps_ed_batch_device_bytes": (_I, [_P, C.POINTER(_U64)]),
    "osmps_ed_batch_set_graph": (_I, [_P, _I]),
    "osmps_ed_batch_set_split": (_I, [_P, _I, _I]),
    "osmps_ed_batch_get_split": (_I, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "osmps_ed_batch_autotune": (_I, [_P, _P, _D, _DP]),
    "osmps_ed_batch_lanczos_ground": (_I, [_P, _P, _D, _P, _P, _P, _P]),
    "osmps_ed_batch_check": (_I, [_P]),
    "osmps_ed_batch_launch_count": (_I, [_P, C.POINTER(C.c_int64)]),
    "osmps_ed_strerror": (C.c_char_p, [_I]),
}


class OsmpsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.osmps_ed_strerror(status).decode() if lib is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libosmps_ed.so not found at {LIB_PATH}; build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    so = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(so, name)
        fn.restype = res
        fn.argtypes = args
    return so


lib = _load()


def check(status: int, where: str, allow=(OSMPS_OK,)):
    if status not in allow:
        raise OsmpsError(status, where)
    return status
