"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/jko.h declares (no compute calls here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(jko_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def libjko():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit to build libjko")
    from paper_1502_06216_gb300 import build
    return ctypes.CDLL(build.build())


def test_every_declared_symbol_is_exported(libjko):
    names = declared_symbols()
    assert {"jko_create", "jko_step", "jko_flow", "jko_destroy"} <= names
    for n in sorted(names):
        assert hasattr(libjko, n), n


def test_binding_covers_header():
    from paper_1502_06216_gb300 import jko
    assert declared_symbols() <= set(jko.EXPORTS)


def test_info_and_status_strings(libjko):
    libjko.jko_status_string.restype = ctypes.c_char_p
    libjko.jko_build_info.restype = ctypes.c_char_p
    assert libjko.jko_status_string(0) == b"JKO_OK"
    assert libjko.jko_status_string(5) == b"JKO_NOT_CONVERGED"
    assert b"sm_103a" in libjko.jko_build_info()


def test_create_rejects_bad_arguments_on_host(libjko):
    """Argument checks happen before any device call."""
    from paper_1502_06216_gb300 import jko
    with pytest.raises(jko.JKOError) as e:
        jko.jko_create(8, 8, gamma=-1.0, tau=0.1, stream=0)
    assert e.value.status == jko.Status.INVALID_ARG
    with pytest.raises(jko.JKOError):
        jko.jko_create(0, 8, gamma=1e-2, tau=0.1, stream=0)
    with pytest.raises(jko.JKOError):
        jko.jko_create(8, 8, gamma=1e-2, tau=0.1, m=0.5, stream=0)


def test_noalloc_step_runs_the_create_checks_on_host(libjko):
    """jko_step_noalloc rejects what jko_create rejects before touching the
    device (its checks are jko_create's): pair_alpha without a second species,
    an unknown species count, non-finite gamma, tau, lengths or exponent.  The
    device pointers are placeholders that are never dereferenced."""
    import math
    from paper_1502_06216_gb300 import jko
    L = jko.lib()
    dummy = ctypes.c_void_p(16)

    def status(grid_kw=None, params_kw=None, energy_kw=None):
        g = jko.jko_grid(8, 8, 1.0, 1.0, 0)
        p = jko.jko_params(1e-2, 0.1, 1e-6, 10, 0, int(jko.Precision.FP32), 1, 0, 0, 0)
        e = jko.jko_energy(None, math.inf, None, 0.0, None, None, None, 0, None, 1, None, 0.0)
        for obj, kw in ((g, grid_kw), (p, params_kw), (e, energy_kw)):
            for k, v in (kw or {}).items():
                setattr(obj, k, v)
        info = jko.jko_step_info()
        return L.jko_step_noalloc(ctypes.byref(g), ctypes.byref(p), ctypes.byref(e), dummy, dummy,
                                  None, ctypes.byref(info))

    bad = [dict(energy_kw=dict(pair_alpha=0.5)),                 # needs species = 2
           dict(energy_kw=dict(species=3)),
           dict(energy_kw=dict(species=-1)),
           dict(params_kw=dict(gamma=math.inf)),
           dict(params_kw=dict(tau=math.inf)),
           dict(params_kw=dict(gamma=-1.0)),
           dict(grid_kw=dict(lx=math.inf)),
           dict(energy_kw=dict(m=math.inf)),
           dict(energy_kw=dict(m=0.5)),
           dict(energy_kw=dict(pair_alpha=math.nan, species=2)),
           dict(params_kw=dict(stall=-1)),
           dict(params_kw=dict(finish=2, stall=4)),
           dict(params_kw=dict(finish=1, stall=4)),                # FP32: no tensor-core pairs
           dict(params_kw=dict(finish=1, stall=0, precision=int(jko.Precision.BF16)))]
    for case in bad:
        assert status(**case) == jko.Status.INVALID_ARG, case
    # limits of the fixed scratch: reported as unsupported, still on the host
    assert status(grid_kw=dict(nx=257)) == jko.Status.UNSUPPORTED
    assert status(params_kw=dict(precision=int(jko.Precision.BF16))) == jko.Status.UNSUPPORTED
