"""CPU checks of the C-ABI library: it builds, loads, exports every function
declared in include/*.h, and its host-side argument checks reject bad input
before touching the device."""
import ctypes
import glob
import os
import re

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_11189_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path)


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^(?!typedef)\s*(?:const\s+)?(?:unsigned\s+|long\s+)*[A-Za-z_]\w*(?:\s+|\s*\*\s*)([A-Za-z_]\w*)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    names.discard("if")
    return sorted(names)


def test_every_declared_function_is_exported(lib):
    names = _declared_functions()
    assert "abacus_flip_ratios" in names and "dysonnet_forward_cache" in names and "local_energy" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2603_11189_gb300 import dysonnet as dn
    assert set(dn.exported_symbols()) <= set(_declared_functions())


def test_status_strings(lib):
    lib.dn_status_string.restype = ctypes.c_char_p
    for s in range(6):
        assert lib.dn_status_string(s).startswith(b"DN_")


class Desc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("L", "d", "s", "w", "d_h", "d_out", "periodic", "f_kind")]


def test_model_create_rejects_bad_descriptors_on_host(lib):
    import numpy as np
    good = synth.ModelDesc(L=2, d=4, s=3, w=1, dh=4, dout=2)
    p = np.zeros(synth.n_params(good))
    h = ctypes.c_void_p()
    bad_descs = [
        Desc(0, 4, 3, 1, 4, 2, 0, 0), Desc(2, 0, 3, 1, 4, 2, 0, 0), Desc(2, 4, 3, -1, 4, 2, 0, 0),
        Desc(2, 4, 3, 1, 4, 9, 0, 0), Desc(2, 4, 3, 1, 4, 2, 2, 0), Desc(2, 4, 3, 1, 4, 2, 0, 5),
        Desc(2, 129, 3, 1, 4, 2, 0, 0),
    ]
    for d in bad_descs:
        assert lib.dn_model_create(ctypes.byref(d), p.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(p.size),
                                   ctypes.byref(h)) == 1
    # wrong parameter count
    d = Desc(2, 4, 3, 1, 4, 2, 0, 0)
    assert lib.dn_model_create(ctypes.byref(d), p.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(p.size - 1),
                               ctypes.byref(h)) == 1
    assert lib.dn_model_create(ctypes.byref(d), None, ctypes.c_size_t(p.size), ctypes.byref(h)) == 1


def test_null_handles_are_rejected(lib):
    lib.dn_cache_bytes.restype = ctypes.c_size_t
    assert lib.dn_cache_bytes(None, 16, 1, 0, 1) == 0
    assert lib.abacus_flip_ratios(None, None, None, 1, None, None) == 1
    assert lib.dysonnet_forward_cache(None, 16, None, 1, 0, 1, None, None, None) == 1
    assert lib.local_energy(None, None, 16, None, 1, 0, None, None) == 1
    assert lib.dn_cache_check(None, None) == 1
    lib.dn_cache_destroy(None)
    lib.dn_model_destroy(None)


def test_parameter_count_matches_generator(lib):
    """The library's layout check agrees with the generator for several shapes
    (DN_EINVAL is returned before any device work only when the count differs)."""
    import numpy as np
    for desc in (synth.CONFIGS["lrtfim_n16"]["desc"], synth.CONFIGS["lrtfim_n128"]["desc"], synth.CONFIGS["j1j2_n256"]["desc"]):
        n = synth.n_params(desc)
        d = Desc(desc.L, desc.d, desc.s, desc.w, desc.dh, desc.dout, desc.periodic, desc.fkind)
        p = np.zeros(n + 1)
        h = ctypes.c_void_p()
        # off by one: rejected on the host
        assert lib.dn_model_create(ctypes.byref(d), p.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n + 1),
                                   ctypes.byref(h)) == 1
