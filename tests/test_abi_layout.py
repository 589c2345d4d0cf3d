"""The Python binding and the C headers describe the same ABI (no GPU).

The binding's ctypes structures must list the header structs' fields in the
same order with the same C types, and its integer constants must equal the
headers' enum values; both are read from the header text, so a change on one
side that the other misses fails here.
"""
import ctypes
import os
import re

import pytest

from paper_2310_04676_gb300 import sg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("sg.h", "sg_ppo.h")]


def _source(path):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return re.sub(r"//[^\n]*", " ", text)


def _struct_fields(name):
    """[(field, kind)] of `typedef struct name {...}` (kind: i32, u32, f32,
    ptr, or (kind, n) for an array)."""
    for path in HEADERS:
        m = re.search(r"typedef\s+struct\s+%s\s*\{(.*?)\}\s*%s\s*;" % (name, name), _source(path),
                      flags=re.S)
        if m:
            break
    else:
        raise AssertionError("struct %s not found" % name)
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.replace("const", " ").strip()
        if not decl:
            continue
        base, rest = decl.split(None, 1)
        kind = {"int32_t": "i32", "uint32_t": "u32", "float": "f32"}[base]
        for d in rest.split(","):
            d = d.strip()
            arr = re.match(r"(\w+)\s*\[(\d+)\]$", d)
            if d.startswith("*"):
                fields.append((d.lstrip("* "), "ptr"))
            elif arr:
                fields.append((arr.group(1), (kind, int(arr.group(2)))))
            else:
                fields.append((d, kind))
    return fields


def _ctypes_kind(t):
    if t is ctypes.c_int32:
        return "i32"
    if t is ctypes.c_uint32:
        return "u32"
    if t is ctypes.c_float:
        return "f32"
    if issubclass(t, (ctypes._Pointer, ctypes.c_void_p)):
        return "ptr"
    if issubclass(t, ctypes.Array):
        return (_ctypes_kind(t._type_), t._length_)
    raise AssertionError("unexpected ctypes type %r" % t)


@pytest.mark.parametrize("cname,pyclass", [("sg_desc", sg.SgDesc), ("sg_plan_info", sg.SgPlanInfo),
                                           ("sg_ppo_config", sg.SgPpoConfig)])
def test_structs_match_the_headers(cname, pyclass):
    want = _struct_fields(cname)
    got = [(n, _ctypes_kind(t)) for n, t in pyclass._fields_]
    assert got == want


def _enum_constants():
    consts = {}
    for path in HEADERS:
        for body in re.findall(r"enum\s*\w*\s*\{(.*?)\}", _source(path), flags=re.S):
            for name, value in re.findall(r"(SG_\w+)\s*=\s*(\d+)", body):
                consts[name] = int(value)
    return consts


# header constants the binding has no use for: joint type codes are written
# into the sg_desc arrays by workloads.py (0 revolute, 1 prismatic), and the
# chain-length limit is checked by the library
HEADER_ONLY = {"SG_JOINT_REVOLUTE", "SG_JOINT_PRISMATIC", "SG_MAX_CHAIN_JOINTS"}


def test_constants_match_the_header_enums():
    consts = _enum_constants()
    assert len(consts) >= 30
    checked = 0
    for name, value in sorted(consts.items()):
        if name in HEADER_ONLY:
            continue
        py = name if hasattr(sg, name) else name[len("SG_"):]
        assert hasattr(sg, py), "binding lacks %s" % name
        assert getattr(sg, py) == value, name
        checked += 1
    assert checked == len(consts) - len(HEADER_ONLY & set(consts))
    # the status names the binding prints are the header's
    for code, text in sg.STATUS_NAMES.items():
        assert consts[text] == code
