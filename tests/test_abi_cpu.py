"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU, exports every
function include/rbe.h declares, and rejects invalid input on the host before any
CUDA call."""
import ctypes as ct

import numpy as np
import pytest

from paper_2609_02694_gb300 import binding, build


@pytest.fixture(scope="module")
def L():
    build.build()
    return binding.lib()


def test_exports_every_declared_function(L):
    names = binding.declared_functions()
    assert "rbe_init" in names and "rbe_forces" in names and "rbe_step" in names
    for n in names:
        assert hasattr(L, n), n
    syms = set()
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", binding.library_path()],
                         capture_output=True, text=True, check=True).stdout
    for line in out.splitlines():
        parts = line.split()
        if parts:
            syms.add(parts[-1])
    assert set(names) <= syms


def test_error_strings(L):
    assert L.rbe_error_string(0) == b"ok"
    assert b"neutral" in L.rbe_error_string(-2)
    assert L.rbe_version().startswith(b"rbe-gb300")


def _params(**kw):
    eps = np.array([0.1])
    sig = np.array([3.0])
    d = dict(alpha=0.09, r_c=10.0, r_core=0.0, p_rbl=10, P=100, seed=1, replica=0,
             precision=0, coulomb_C=332.06371, dt=1.0, kappa=4.184e-4, n_types=1,
             lj_eps=eps.ctypes.data_as(ct.POINTER(ct.c_double)),
             lj_sigma=sig.ctypes.data_as(ct.POINTER(ct.c_double)), cell_sub=0)
    d.update(kw)
    return binding.Params(**d), (eps, sig)


def _init(L, p, N=4, L_box=32.0, q=None):
    box = np.array([L_box] * 3)
    pos = np.random.default_rng(0).uniform(0, L_box, (N, 3))
    q = np.array([1.0, -1.0, 1.0, -1.0][:N]) if q is None else np.asarray(q, float)
    h = ct.c_void_p()
    rc = L.rbe_init(ct.byref(h), ct.byref(p), N, box.ctypes.data, pos.ctypes.data,
                    q.ctypes.data, None, None, None, None)
    return rc, h


def test_host_validation_before_cuda(L):
    p, keep = _params()
    assert _init(L, p, q=[1.0, 1.0, -1.0, 0.5])[0] == -2         # not neutral
    p2, keep2 = _params(r_c=16.5)
    assert _init(L, p2)[0] == -3                                 # r_c >= L/2
    p3, keep3 = _params(P=0)
    assert _init(L, p3)[0] == -1
    p4, keep4 = _params(r_core=12.0)
    assert _init(L, p4)[0] == -1                                 # r_core >= r_c
    p5, keep5 = _params(r_core=5.0, r_c=12.0)
    assert _init(L, p5, L_box=30.0)[0] == -4                     # RBL needs 3 cells of r_s
    p6, keep6 = _params(precision=7)
    assert _init(L, p6)[0] == -1
    h = ct.c_void_p()
    assert L.rbe_init(None, ct.byref(p), 4, None, None, None, None, None, None, None) == -1
    assert L.rbe_destroy(None) == 0
