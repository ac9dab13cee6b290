"""The Python binding's view of the C ABI, checked against include/mpt.h
itself: a C program compiled with the host compiler against the header
prints the size and every field offset of each argument struct and the value
of each constant, and they must equal the ctypes structures and the
constants the binding (and the scene builder) use.  A field added, dropped
or reordered on one side only would otherwise pass wrong values through
the boundary without an error."""
import ctypes as C
import json
import os
import shutil
import subprocess

import pytest

from paper_2301_06399_gb300 import mpt
from paper_2301_06399_gb300 import scenes as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "mpt_scene_desc": mpt.SceneDesc,
    "mpt_endpoints": mpt.Endpoints,
    "mpt_sampling": mpt.Sampling,
    "mpt_candidates": mpt.CandStruct,
    "mpt_solutions": mpt.SolStruct,
    "mpt_schedule": mpt.Schedule,
    "mpt_paths": mpt.PathStruct,
    "mpt_field_params": mpt.FieldParams,
}

CONSTANTS = {
    "MPT_OK": mpt.MPT_OK, "MPT_ERR_ARG": mpt.MPT_ERR_ARG, "MPT_ERR_CUDA": mpt.MPT_ERR_CUDA,
    "MPT_ERR_CAPACITY": mpt.MPT_ERR_CAPACITY, "MPT_ERR_TIMEOUT": mpt.MPT_ERR_TIMEOUT,
    "MPT_ERR_UNSUPPORTED": mpt.MPT_ERR_UNSUPPORTED,
    "MPT_FP64_PLAIN": mpt.FP64_PLAIN, "MPT_FP32": mpt.FP32, "MPT_FP32_FP64REFINE": mpt.FP32_FP64REFINE,
    "MPT_PATH_CONVERGED": mpt.PATH_CONVERGED, "MPT_PATH_MAXITER": mpt.PATH_MAXITER,
    "MPT_PATH_DIVERGED": mpt.PATH_DIVERGED, "MPT_PATH_STALLED": mpt.PATH_STALLED,
    "MPT_PATH_NONFINITE": mpt.PATH_NONFINITE, "MPT_PATH_EXCLUDED": mpt.PATH_EXCLUDED,
    "MPT_PATH_REFINED": mpt.PATH_REFINED, "MPT_PATH_PRESCREENED": mpt.PATH_PRESCREENED,
    "MPT_PATH_FALLBACK": mpt.PATH_FALLBACK,
    "MPT_PLANE": S.PLANE, "MPT_PARABOLOID": S.PARABOLOID, "MPT_LINE_EDGE": S.LINE_EDGE,
    "MPT_ARC_EDGE": S.ARC_EDGE, "MPT_OCC_RECT": S.OCC_RECT, "MPT_OCC_PARABOLOID": S.OCC_PARABOLOID,
    "MPT_RECORD": S.REC, "MPT_MAX_ORDER": len(mpt.Sampling().quota),
}


def _program() -> str:
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mpt.h"', "int main(void) {",
             '  printf("{");']
    first = True
    for name, cls in STRUCTS.items():
        sep = "" if first else ","
        first = False
        lines.append(f'  printf("{sep}\\"{name}\\": {{\\"size\\": %zu", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf(", \\"{field}\\": %zu", offsetof({name}, {field}));')
        lines.append('  printf("}");')
    for name in CONSTANTS:
        lines.append(f'  printf(", \\"{name}\\": %lld", (long long)({name}));')
    lines += ['  printf("}\\n");', "  return 0;", "}"]
    return "\n".join(lines) + "\n"


@pytest.fixture(scope="module")
def header_view(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text(_program())
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    return json.loads(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)


@pytest.mark.parametrize("name", sorted(STRUCTS))
def test_struct_layout_matches_the_header(header_view, name):
    cls = STRUCTS[name]
    got = header_view[name]
    assert got["size"] == C.sizeof(cls), (name, got["size"], C.sizeof(cls))
    for field, _ in cls._fields_:
        assert got[field] == getattr(cls, field).offset, (name, field, got[field], getattr(cls, field).offset)


def test_every_header_struct_is_bound():
    text = open(os.path.join(ROOT, "include", "mpt.h")).read()
    import re

    declared = set(re.findall(r"\}\s*(mpt_[a-z_]+)\s*;", text))
    assert declared == set(STRUCTS), declared ^ set(STRUCTS)


def test_constants_match_the_header(header_view):
    for name, value in CONSTANTS.items():
        assert header_view[name] == value, (name, header_view[name], value)
