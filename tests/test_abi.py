"""The C ABI library builds, loads on a machine without a GPU, and exports
every entry point that include/harmrad.h declares; the Python parameter
struct matches the header field by field.  No kernel is called here."""
import ctypes
import os
import re

import pytest

from paper_1312_6127_gb300 import _build
from paper_1312_6127_gb300 import harmrad as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "harmrad.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(harmrad_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = _build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(H.EXPORTS) == names


def test_params_struct_matches_header():
    text = open(HEADER).read()
    body = text[text.index("typedef struct harmrad_params {"):text.index("} harmrad_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for line in body.splitlines()[1:]:
        line = line.strip().rstrip(";")
        if not line:
            continue
        typ, rest = line.split(None, 1)
        for f in rest.split(","):
            f = f.strip()
            fields.append(f.split("[")[0])
    assert fields == [name for name, _ in H.Params._fields_]


def test_strerror_without_gpu(lib):
    lib.harmrad_strerror.restype = ctypes.c_char_p
    assert b"invalid" in lib.harmrad_strerror(-1)
    assert lib.harmrad_strerror(0) == b"ok"


def test_invalid_params_rejected_on_host(lib):
    """Argument validation happens on the host before any device call."""
    from paper_1312_6127_gb300 import workloads as W
    cfg, _ = W.relax_box(n1=16)
    bad = dict(cfg, newton_max=0)
    p = H.make_params(bad)
    L = H.load(_build.LIB)
    rc = L.harmrad_zone_physics(ctypes.byref(p), 0, None, None, None, None, None, None, None)
    assert rc == -1
    ok = H.make_params(cfg)
    assert L.harmrad_zone_physics(ctypes.byref(ok), 0, None, None, None, None, None, None, None) == 0
    polar_bad = dict(cfg, bc=[0, 0, 2, 2, 0, 0])  # polar axis needs the Kerr-Schild metric
    assert L.harmrad_zone_physics(ctypes.byref(H.make_params(polar_bad)), 0, None, None, None, None,
                                  None, None, None) == -1
    for over, rc in ((dict(integrator=3), 0), (dict(integrator=4), -1), (dict(integrator=-1), -1),
                     (dict(bc=[3, 3, 0, 0, 0, 0]), 0), (dict(bc=[4, 4, 0, 0, 0, 0]), 0),
                     (dict(bc=[5, 5, 0, 0, 0, 0]), -1)):
        q = H.make_params(dict(cfg, **over))
        assert L.harmrad_zone_physics(ctypes.byref(q), 0, None, None, None, None, None, None, None) == rc, over
