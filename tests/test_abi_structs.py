"""The Python binding's ctypes structures mirror the C structs of
include/amg_gb300.h field by field (name, order, scalar type and array
length), so that adding a field on one side only fails on the CPU."""
import ctypes
import os
import re

from paper_2511_21268_gb300 import amg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_TYPES = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
           "double": ctypes.c_double}


def header_fields(name):
    src = open(os.path.join(ROOT, "include", "amg_gb300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    out = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        mm = re.match(r"(?:const )?([A-Za-z_0-9]+) ?(\**) ?([A-Za-z_0-9]+)(?:\[([A-Za-z_0-9]+)\])?$", decl)
        assert mm, decl
        typ, ptr, field, arr = mm.groups()
        n = None if arr is None else (int(arr) if arr.isdigit() else getattr(amg, arr))
        out.append((field, typ, bool(ptr), n))
    return out


def check(cstruct, pystruct):
    want = header_fields(cstruct)
    got = pystruct._fields_
    assert [f for f, *_ in want] == [f for f, _ in got], cstruct
    for (field, typ, is_ptr, n), (_, ct) in zip(want, got):
        if is_ptr:
            assert ct in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(ct, "contents"), (cstruct, field)
            continue
        if n is not None:
            assert issubclass(ct, ctypes.Array) and ct._length_ == n, (cstruct, field)
            ct = ct._type_
        assert ct is C_TYPES[typ], (cstruct, field, typ, ct)


def test_opts_struct_mirrors_header():
    check("amg_opts", amg.AmgOpts)


def test_info_struct_mirrors_header():
    check("amg_info", amg.AmgInfo)


def test_csr_struct_mirrors_header():
    check("amg_csr", amg.AmgCsr)


def test_documented_option_defaults_are_the_defaults():
    """Each amg_opts field's header comment ends with its default in
    parentheses; amg_opts_default (host only) must fill exactly those."""
    from paper_2511_21268_gb300 import _build

    src = open(os.path.join(ROOT, "include", "amg_gb300.h")).read()
    body = re.search(r"typedef struct \{([^{}]*)\}\s*amg_opts\s*;", src).group(1)
    documented = {}
    for m in re.finditer(r"([A-Za-z_0-9 \*]+?)\s*;\s*/\*(.*?)\*/", body, flags=re.S):
        field = m.group(1).split()[-1].lstrip("*")
        default = re.findall(r"\(([^()]*)\)\s*$", " ".join(m.group(2).split()))
        assert default, field
        documented[field] = default[0]
    assert set(documented) == {f for f, _ in amg.AmgOpts._fields_}
    L = ctypes.CDLL(_build.build_cuda())
    o = amg.AmgOpts()
    assert L.amg_opts_default(ctypes.byref(o)) == 0
    for field, text in documented.items():
        got = getattr(o, field)
        if text == "NULL":
            assert got is None, field
        elif text.startswith("AMG_"):
            assert got == getattr(amg, text), field
        else:
            assert got == type(got)(float(text) if "." in text else int(text)), (field, got, text)


def test_iga_patch_struct_mirrors_header():
    check("amg_iga_patch", amg.AmgIgaPatch)
