"""The C-ABI library loads without a GPU and exports every declared call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(adr_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libadr():
    from paper_2411_11041_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_library_exports_every_declared_call(libadr):
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(libadr, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_2411_11041_gb300 as P
    assert sorted(P.EXPORTED) == [n for n in declared_functions() if n in P.EXPORTED]
    for n in P.EXPORTED:
        assert n in declared_functions()


def test_default_opts_without_gpu(libadr):
    import paper_2411_11041_gb300 as P
    o = P.default_opts()
    assert o.theta == 0.5 and o.tol == 1e-10 and o.prec == P.ADR_FP64


def test_create_rejects_bad_arguments_without_touching_the_gpu(libadr):
    import paper_2411_11041_gb300 as P
    g = P.adr_grid(2, 5, 0.0, 0.0, 1.0, 1.0)
    o = P.default_opts()
    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    st = P.lib().adr_create(ctypes.byref(g), dummy, 1.0, 1.0, dummy, dummy, dummy, ctypes.byref(o),
                            None, ctypes.byref(h))
    assert st == P.ADR_EINVAL and b"nx" in P.lib().adr_last_error()
    g = P.adr_grid(8, 8, 0.0, 0.0, 1.0, 1.0)
    st = P.lib().adr_create(ctypes.byref(g), dummy, -1.0, 1.0, dummy, dummy, dummy, ctypes.byref(o),
                            None, ctypes.byref(h))
    assert st == P.ADR_EINVAL
    o.theta = 0.0
    st = P.lib().adr_create(ctypes.byref(g), dummy, 1.0, 1.0, dummy, dummy, dummy, ctypes.byref(o),
                            None, ctypes.byref(h))
    assert st == P.ADR_EINVAL and b"theta" in P.lib().adr_last_error()
    o.theta = 0.5
    o.transfer = 2
    st = P.lib().adr_create(ctypes.byref(g), dummy, 1.0, 1.0, dummy, dummy, dummy, ctypes.byref(o),
                            None, ctypes.byref(h))
    assert st == P.ADR_EINVAL and b"transfer" in P.lib().adr_last_error()
    o.transfer, o.prec = 1, P.ADR_FP32_REFINE  # the direct transfer runs in FP64 only
    st = P.lib().adr_create(ctypes.byref(g), dummy, 1.0, 1.0, dummy, dummy, dummy, ctypes.byref(o),
                            None, ctypes.byref(h))
    assert st == P.ADR_EINVAL and b"transfer" in P.lib().adr_last_error()


def test_network_parameter_layout_without_gpu(libadr):
    """The seeded initial parameters have the library's parameter count, and
    the binding refuses a vector of another length before any copy."""
    import numpy as np

    import paper_2411_11041_gb300 as P
    from paper_2411_11041_gb300 import workloads as W
    ch = W.CNN_CHANNELS
    assert P.adr_cnn_num_params() == sum(9 * a * b + b for a, b in zip(ch[:-1], ch[1:]))
    assert W.cnn_init_params().size == P.adr_cnn_num_params()
    with pytest.raises(ValueError):
        P.adr_cnn_create(1, np.zeros(10, np.float32))


def _header_struct_fields(name):
    src = open(os.path.join(ROOT, "include", "adr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", src).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, rest = decl.split(None, 1)
        for nm in rest.split(","):
            fields.append((ctype, nm.strip()))
    return fields


@pytest.mark.parametrize("name", ["adr_stats", "adr_opts", "adr_grid"])
def test_binding_structs_match_header(name):
    """The ctypes mirrors have the header's fields, in order, with the same C types."""
    import paper_2411_11041_gb300 as P
    want = _header_struct_fields(name)
    got = getattr(P, name)._fields_
    ctypes_of = {"int": ctypes.c_int, "double": ctypes.c_double}
    assert [n for _, n in want] == [n for n, _ in got]
    assert [ctypes_of[t] for t, _ in want] == [t for _, t in got]
