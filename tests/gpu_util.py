"""Shared helpers for the GPU parity tests."""
import os

import numpy as np

TOL_C128 = 1e-12          # max-abs, complex128
TOL_C64 = 1e-5            # max-abs, complex64
TOL_C64_INFIDELITY = 1e-8  # 1 - |<oracle|gpu>|^2 / (|oracle|^2 |gpu|^2), complex64


def compare(got: np.ndarray, ref: np.ndarray, piece: int = 1 << 24):
    """(max |got - ref|, 1 - fidelity) in FP64, in pieces so huge states need no temporaries."""
    assert got.shape == ref.shape
    mx = 0.0
    ov = 0j
    ng = 0.0
    nr = 0.0
    for s in range(0, got.size, piece):
        g = got[s:s + piece].astype(np.complex128)
        r = ref[s:s + piece]
        mx = max(mx, float(np.abs(g - r).max()))
        ov += np.vdot(r, g)
        ng += float(np.vdot(g, g).real)
        nr += float(np.vdot(r, r).real)
    return mx, 1.0 - abs(ov) ** 2 / (ng * nr)


def assert_close(got, ref, dtype):
    mx, inf = compare(got, ref)
    if dtype == "c128":
        assert mx <= TOL_C128, f"max-abs {mx:.3e} > {TOL_C128}"
    else:
        assert mx <= TOL_C64, f"max-abs {mx:.3e} > {TOL_C64}"
        assert inf <= TOL_C64_INFIDELITY, f"1-F {inf:.3e} > {TOL_C64_INFIDELITY}"
    return mx, inf


def host_ram_bytes() -> int:
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        return 0
