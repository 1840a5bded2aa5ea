"""The C-ABI library loads and exports every entry point include/lsq.h declares.

No compute call is made (there may be no GPU here)."""
import ctypes
import os
import re

import pytest

import paper_2002_07704_gb300 as lsq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^int\s+(lsq_\w+)\s*\(", txt, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    lsq.build()
    return ctypes.CDLL(lsq.library_path())


def test_header_declares_the_paths_calls():
    d = _declared()
    for name in ("lsq_build_neighbour_lists", "lsq_block_matmul", "lsq_lnv_energy_gradient",
                 "lsq_lnv_minimise"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    assert set(lsq.exported_symbols()) == _declared()


def test_host_only_calls(lib):
    lsq.load()
    assert lsq.load().lsq_version() == 100
    out = (ctypes.c_double * 6)()
    assert lsq.load().lsq_lnv_required_ranges(6.6, 6.6, 10.0, out) == 0
    assert list(out) == [6.6, 6.6, 10.0, 10.0 + 6.6, 10.0 + 6.6 + 10.0, 6.6 + 10.0 + 6.6]
    o = lsq.LnvOpts()
    assert lsq.load().lsq_lnv_default_opts(ctypes.byref(o)) == 0
    assert o.cg_reset == 40 and o.spin == 2.0


def test_invalid_arguments_are_rejected_without_gpu(lib):
    L = lsq.load()
    h = ctypes.c_void_p()
    # null output handle, bad range count, non-positive range: all rejected on the host
    assert L.lsq_build_neighbour_lists(None, 0, None, None, 0, None, None) == 1
    cell = (ctypes.c_double * 3)(10.0, 10.0, 10.0)
    rng = (ctypes.c_double * 1)(-1.0)
    assert L.lsq_build_neighbour_lists(None, 0, cell, rng, 1, ctypes.byref(h), None) == 1
    buf = ctypes.create_string_buffer(256)
    assert L.lsq_last_error(buf, 256) == 1 and b"positive" in buf.value
    assert L.lsq_block_matmul(None, 4, 0, 0, 0, None, 0, 0, None, 0, None, 1.0, 0.0, None, None) == 1


def test_binding_rejects_wrong_sizes_without_gpu():
    """Every matrix argument must hold exactly nnzb(range) b x b values; a short (or long)
    tensor raises LsqError(INVALID_ARG) on the host, before any device call."""
    import torch

    class FakeGeom:
        handle = None

        def nnzb(self, r):
            return {0: 10, 1: 7}[r]

    A = torch.zeros(10 * 16)
    short = torch.zeros(7 * 16 - 1)
    with pytest.raises(lsq.LsqError) as e:
        lsq.block_matmul(FakeGeom(), 4, A, 0, A, 0, short, 1)
    assert e.value.code == 1 and "C has 111 values" in str(e.value)
    with pytest.raises(lsq.LsqError) as e:
        lsq.trace(FakeGeom(), 4, A, 0, torch.zeros(8 * 16), 1)
    assert e.value.code == 1
    with pytest.raises(lsq.LsqError) as e:
        lsq.transpose(FakeGeom(), 13, torch.zeros(10 * 169), 0, torch.zeros(7 * 16), 1)
    assert e.value.code == 1


def _prototypes():
    """{name: [parameter kind]} of every entry point of include/*.h: 'ptr', 'int', 'i64',
    'size' or 'double' (the opaque handles lsq_geom and lsq_lnv are pointers)."""
    out = {}
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
        for name, params in re.findall(r"^int\s+(lsq_\w+)\s*\(([^;]*?)\)\s*;", txt, flags=re.M | re.S):
            kinds = []
            for p in [q.strip() for q in params.split(",")]:
                if p in ("", "void"):
                    continue
                words = p.replace("const ", "").split()
                if "*" in p or words[0] in ("lsq_geom", "lsq_lnv"):
                    kinds.append("ptr")
                else:
                    kinds.append({"int": "int", "int64_t": "i64", "size_t": "size", "double": "double"}[words[0]])
            out[name] = kinds
    return out


def test_binding_argtypes_match_the_header(lib):
    """Every ctypes signature the binding sets has the header's parameter count and kinds, so no
    argument is passed with the wrong width."""
    kind = {ctypes.c_void_p: "ptr", ctypes.c_char_p: "ptr", ctypes.c_int: "int", ctypes.c_int64: "i64",
            ctypes.c_size_t: "size", ctypes.c_double: "double"}
    L = lsq.load()
    protos = _prototypes()
    assert set(protos) == _declared()
    for name, params in protos.items():
        got = [kind[t] for t in getattr(L, name).argtypes]
        assert got == params, name
