"""The library's host test entries (include/psc_testing.h): the kernels' own helper
functions compiled for the host, loaded through ctypes. No GPU is needed."""
import ctypes as C

import pytest

_L = None


def lib():
    global _L
    if _L is None:
        from paper_1901_09745_gb300 import build
        build.build()
        import paper_1901_09745_gb300 as P
        L = C.CDLL(P.library_path())
        ip, dp = C.POINTER(C.c_int), C.POINTER(C.c_double)
        sig = {
            "psc_test_axis_tile_ranges": ([C.c_int] * 6 + [ip, ip], C.c_int),
            "psc_test_axis_tile": ([C.c_int, C.c_int, ip, ip], C.c_int),
            "psc_test_tile_in_reach": ([dp, C.c_double, ip, ip, ip, ip, C.c_int], C.c_int),
            "psc_test_record_rel": ([C.c_double, C.c_int, C.c_int, C.c_int, C.c_int], C.c_float),
            "psc_test_axis_span": ([C.c_int, C.c_int, C.c_int, ip, ip], None),
            "psc_test_axis_at": ([C.c_int] * 4, C.c_int),
            "psc_test_contact_sign": ([C.c_double, C.c_double, ip, ip], C.c_int),
            "psc_test_jkr_s": ([C.c_float, C.c_float, ip, ip], C.c_float),
            "psc_test_moved2": ([dp, dp, ip, ip, C.c_int], C.c_float),
            "psc_test_all_finite": ([C.c_void_p, C.c_longlong], C.c_int),
            "psc_test_radii_range": ([C.c_void_p, C.c_int, dp, dp], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes, fn.restype = args, res
        _L = L
    return _L


@pytest.fixture(scope="module")
def H():
    return lib()


def ints(*v):
    return (C.c_int * len(v))(*[int(x) for x in v])


def doubles(*v):
    return (C.c_double * len(v))(*[float(x) for x in v])
