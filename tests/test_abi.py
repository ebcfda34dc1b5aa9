"""The C-ABI library loads and exports what include/parament.h declares; host-only logic.

No compute calls here: these run without a GPU.
"""

import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "parament.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(parament_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("parament_create", "parament_destroy", "parament_set_hamiltonians", "parament_set_controls",
                     "parament_propagate"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2108_07126_gb300 import binding

    lib = ctypes.CDLL(binding.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert binding.parament_version() == 1


def test_status_strings():
    from paper_2108_07126_gb300 import binding as b

    assert b.parament_status_string(b.PARAMENT_OK) == "PARAMENT_OK"
    assert b.parament_status_string(b.PARAMENT_ERR_STATE) == "PARAMENT_ERR_STATE"
    assert b.parament_status_string(12345) == "PARAMENT_UNKNOWN_STATUS"


def test_null_arguments_are_rejected_without_a_device():
    from paper_2108_07126_gb300 import binding as b

    assert b.raw_call("parament_destroy", None) == b.PARAMENT_OK
    assert b.raw_call("parament_create", None, 0, None) == b.PARAMENT_ERR_INVALID_VALUE
    assert b.raw_call("parament_propagate", None, None, 0) == b.PARAMENT_ERR_INVALID_VALUE
    assert b.raw_call("parament_set_option", None, 1, 0) == b.PARAMENT_ERR_INVALID_VALUE


def test_create_without_gpu_reports_cuda_error():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2108_07126_gb300 import binding as b

    h = ctypes.c_void_p()
    assert b.raw_call("parament_create", ctypes.byref(h), 0, None) == b.PARAMENT_ERR_CUDA
    assert not h.value


@pytest.mark.parametrize("m", [1, 2, 4, 6, 9, 12, 16, 20])
@pytest.mark.parametrize("u", [2.0 ** -53, 2.0 ** -24])
def test_taylor_theta_solves_the_remainder_bound(m, u):
    """theta_m is the root of x^(m+1)/(m+1)! e^x = u, checked with 50-digit arithmetic."""
    import mpmath

    from paper_2108_07126_gb300 import binding as b

    mpmath.mp.dps = 50
    th = b.parament_taylor_theta(m, u)
    f = lambda x: (m + 1) * mpmath.log(x) - mpmath.log(mpmath.factorial(m + 1)) + x - mpmath.log(u)
    ref = mpmath.findroot(f, (mpmath.mpf("1e-30"), mpmath.mpf(50)), solver="illinois")
    assert abs(th - float(ref)) <= 1e-12 * float(ref)
    # monotone in m
    assert b.parament_taylor_theta(m + 1, u) > th


def test_taylor_theta_invalid():
    from paper_2108_07126_gb300 import binding as b

    assert b.parament_taylor_theta(0, 1e-16) < 0
    assert b.parament_taylor_theta(3, 0.0) < 0


PS_PRODUCTS = {1: 0, 2: 1, 4: 2, 6: 3, 9: 4, 12: 5}


def brute_choice(nu, u, force_m=0):
    """Cheapest (m, s) with nu / 2^s <= theta_m(u / 2^s), by enumeration in 50-digit arithmetic."""
    import mpmath

    mpmath.mp.dps = 50
    best = None
    for s in range(0, 63):
        for m, cost in PS_PRODUCTS.items():
            if force_m and m != force_m:
                continue
            x = mpmath.mpf(nu) / mpmath.mpf(2) ** s
            ok = x == 0 or (m + 1) * mpmath.log(x) - mpmath.log(mpmath.factorial(m + 1)) + x <= mpmath.log(
                mpmath.mpf(u) / mpmath.mpf(2) ** s)
            if ok and (best is None or cost + s < best[0]):
                best = (cost + s, m, s)
    return best[1], best[2]


@pytest.mark.parametrize("nu", [0.0, 1e-12, 1e-5, 0.01, 0.13, 0.16, 0.4, 1.0, 3.9, 12.0, 250.0])
@pytest.mark.parametrize("u", [2.0 ** -53, 2.0 ** -24])
def test_taylor_choice_is_cheapest_admissible(nu, u):
    from paper_2108_07126_gb300 import binding as b

    m, s = b.parament_taylor_choice(nu, u)
    bm, bs = brute_choice(nu, u)
    assert PS_PRODUCTS[m] + s == PS_PRODUCTS[bm] + bs
    # admissible: the bound holds at the chosen pair
    assert nu / 2 ** s <= b.parament_taylor_theta(m, u / 2 ** s) * (1 + 1e-12)


def test_taylor_choice_forced_and_invalid():
    from paper_2108_07126_gb300 import binding as b

    for m in (4, 6, 9, 12):
        mm, s = b.parament_taylor_choice(0.5, 2.0 ** -53, m)
        assert mm == m and (m, s) == brute_choice(0.5, 2.0 ** -53, m)
    with pytest.raises(b.ParamentError):
        b.parament_taylor_choice(0.5, 2.0 ** -53, 5)
    with pytest.raises(b.ParamentError):
        b.parament_taylor_choice(float("nan"), 2.0 ** -53)


def test_chebyshev_bound_reproduces_table1():
    """Table 1 of Sec. 2.1 from the error bound of Eq. error_chebychev (printed to three digits)."""
    import json

    from paper_2108_07126_gb300 import binding as b

    t = json.load(open(os.path.join(ROOT, "tests", "golden", "chebyshev_table1.json")))
    for m, v32, v64 in zip(t["m_max"], t["fp32"], t["fp64"]):
        th32 = b.parament_chebyshev_theta(m, 2.0 ** -24)
        th64 = b.parament_chebyshev_theta(m, 2.0 ** -53)
        assert abs(th32 - v32) <= 0.5e-3 + 1e-9, (m, th32, v32)
        if m == 3:
            assert abs(th64 - v64) <= 0.5e-4, (m, th64)  # printed as 2e-4
        else:
            assert abs(th64 - v64) <= 0.5e-3 + 1e-9, (m, th64, v64)
        assert b.parament_chebyshev_degree(th32 * 0.999, 2.0 ** -24) <= m
        assert b.parament_chebyshev_degree(th32 * 1.001, 2.0 ** -24) > m


@pytest.mark.parametrize("x", [0.0, 1e-8, 0.3, 1.7, 4.45, 9.9, 25.0])
def test_bessel_sequence_matches_scipy(x):
    import scipy.special

    from paper_2108_07126_gb300 import binding as b

    n = 40
    got = b.parament_bessel_j(n, x)
    ref = scipy.special.jv(range(n + 1), x)
    assert max(abs(g - r) for g, r in zip(got, ref)) <= 1e-14
