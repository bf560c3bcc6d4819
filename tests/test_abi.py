"""The C-ABI library: it builds, loads, exports every symbol the header declares, and its
host-only logic (the irreducible q set) matches the oracle bit for bit.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import phx_inputs as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            text = open(os.path.join(ROOT, "include", name)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            syms |= set(re.findall(r"\b(phx_[a-z0-9_]+)\s*\(", text))
    return syms


@pytest.fixture(scope="module")
def phx():
    lib = os.path.join(ROOT, "paper_2602_23728_gb300", "libphx.so")
    if not os.path.exists(lib):
        import __graft_entry__
        __graft_entry__.build()
    import paper_2602_23728_gb300 as m
    return m


def test_library_exports_every_declared_symbol(phx):
    lib = ctypes.CDLL(phx.LIB_PATH)
    declared = _declared_symbols()
    assert len(declared) >= 12
    for s in sorted(declared):
        assert hasattr(lib, s), f"{s} declared in include/ but not exported"
    assert set(phx.EXPORTED) <= declared


def test_version_string(phx):
    assert "sm_103a" in phx.version()


@pytest.mark.parametrize("mesh,which", [((5, 5, 5), "oh1"), ((8, 8, 8), "tr"), ((4, 6, 5), "tr"),
                                        ((8, 8, 8), "oh4"), ((24, 24, 24), "oh4"), ((1, 1, 1), "tr")])
def test_irreducible_matches_oracle(phx, mesh, which):
    if which == "oh1":
        rots = P.cubic_rotations_reduced(P.fcc_primitive().lattice)
    elif which == "oh4":
        rots = P.cubic_rotations_reduced(P.fcc_conventional().lattice)
    else:
        rots = P.identity_rotation()
    irr, f2i, wt = phx.irreducible(mesh, rots)
    oirr, of2i, owt = O.grid.irreducible(mesh, rots)
    assert np.array_equal(irr, oirr)
    assert np.array_equal(f2i, of2i)
    assert np.array_equal(wt, owt)


@pytest.mark.parametrize("mesh", [(1, 1, 1), (2, 2, 2), (3, 3, 3), (4, 2, 2), (5, 4, 3), (8, 8, 8)])
def test_time_reversal_count_sizes_the_bte_unknowns(phx, mesh):
    """The binding sizes phx_kappa_sc's outputs by the number of orbits {q, -q}: equal to the
    oracle's time-reversal set and to the library's irreducible set without rotations."""
    irr, _, _ = O.bte.time_reversal_set(mesh)
    lib_irr, _, _ = phx.irreducible(mesh, P.identity_rotation())
    assert phx.time_reversal_count(mesh) == len(irr) == len(lib_irr)
    assert np.array_equal(irr, lib_irr)


def test_irreducible_rejects_incompatible_rotation(phx):
    rot = np.array([[[0, 1, 0], [1, 0, 0], [0, 0, 1]]], dtype=np.int32)   # swaps axes of a 4x6 mesh
    with pytest.raises(phx.PhxError):
        phx.irreducible((4, 6, 5), rot)


def test_create_without_gpu_fails_loudly(phx):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(phx.PhxError):
        phx.Context(0)


def _header_structs():
    """Field lists (name, C type) of the typedef'd structs of the header, in order."""
    text = ""
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            text += open(os.path.join(ROOT, "include", name)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, tag in re.findall(r"typedef struct\s*\{(.*?)\}\s*(phx_[a-z0-9_]+)\s*;", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"(.*?)([A-Za-z_][A-Za-z0-9_]*)\s*(\[\s*(\d+)\s*\])?$", decl)
            ctype = m.group(1).replace("const ", "").strip()
            fields.append((m.group(2), ctype, int(m.group(4)) if m.group(4) else None))
        out[tag] = fields
    return out


@pytest.mark.parametrize("tag,cls", [("phx_cell", "Cell"), ("phx_ifc2", "Ifc2"), ("phx_ifc3", "Ifc3"),
                                     ("phx_broadening", "Broadening"), ("phx_job", "Job"), ("phx_tune", "Tune")])
def test_ctypes_structs_mirror_the_header(phx, tag, cls):
    """The binding's ctypes mirrors of the ABI structs have the header's fields, in order and
    with matching C types (pointer, int32, int64, double, nested struct, fixed array)."""
    import paper_2602_23728_gb300._lib as L
    structs = _header_structs()
    assert tag in structs
    mirror = getattr(L, cls)._fields_
    assert [f[0] for f in mirror] == [f[0] for f in structs[tag]]
    scalar = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double}
    for (name, ctype, count), (mname, mtype) in zip(structs[tag], mirror):
        if ctype.endswith("*"):
            assert mtype is ctypes.c_void_p, (tag, name)
        elif count is not None:
            assert mtype == scalar[ctype] * count, (tag, name)
        elif ctype in scalar:
            assert mtype is scalar[ctype], (tag, name)
        else:                                           # nested struct by value
            assert ctype.startswith("phx_") and mtype.__name__ == {"phx_broadening": "Broadening"}[ctype], (tag, name)
