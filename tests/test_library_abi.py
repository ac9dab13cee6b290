"""The C-ABI library without a GPU: it builds, loads, exports every symbol
include/mpt.h declares, and its host-only entry points behave."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2301_06399_gb300 import build

    build.build()
    from paper_2301_06399_gb300 import mpt

    return mpt.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mpt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpt_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    from paper_2301_06399_gb300 import mpt

    assert sorted(mpt.SYMBOLS) == names


def test_status_strings(lib):
    from paper_2301_06399_gb300 import mpt

    for rc in range(6):
        assert mpt.status_string(rc).startswith("MPT_")
    assert "CAPACITY" in mpt.status_string(mpt.MPT_ERR_CAPACITY)


def _chol_solve_flops(q: int) -> int:
    """Operation count of the packed Cholesky + two triangular solves as
    written in the kernel: column j costs 2j (dot) + 3 (diagonal update with
    relative damping), each entry below it 2j + 1; the solves cost 2i + 1 and
    2(q-1-i) + 1 per row."""
    f = 0
    for j in range(q):
        f += 2 * j + 3
        f += (q - 1 - j) * (2 * j + 1)
    for i in range(q):
        f += 2 * i + 1
        f += 2 * (q - 1 - i) + 1
    return f


@pytest.mark.parametrize("kinds", [[0], [2], [0, 0], [0, 2], [2, 2], [0, 0, 0], [2, 0, 2, 0], [1], [3], [1, 3]])
def test_flop_model_counts(lib, kinds):
    from paper_2301_06399_gb300 import mpt

    f_iter, f_eval, sfu = mpt.flop_model(kinds)
    # the factorisation runs over the live parameters: two per surface
    # interaction, one per edge
    live = sum(1 if k in (2, 3) else 2 for k in kinds)
    assert f_iter == _chol_solve_flops(live)
    assert f_eval > 50 * len(kinds)
    # one reciprocal square root per segment, one more per paraboloid normal,
    # two sin/cos pairs per arc (point and tangent; 2 SFU operations each)
    n = len(kinds)
    assert sfu == (n + 1) + kinds.count(1) + 4 * kinds.count(3)


def test_flop_model_rejects_bad_arguments(lib):
    from paper_2301_06399_gb300 import mpt

    with pytest.raises(RuntimeError):
        mpt.flop_model([0, 0, 0, 0, 0])
    with pytest.raises(RuntimeError):
        mpt.flop_model([7])


def test_null_arguments_are_rejected_without_a_gpu(lib):
    # argument checks run on the host before any CUDA call
    assert lib.mpt_scene_upload(None, None, None) == 1
    assert lib.mpt_solve(None, None, None, None, 0, None, None, None) == 1
    assert lib.mpt_validate(None, None, None, None, None, C.c_double(1e-20), None, None, None) == 1
    assert lib.mpt_grad(None, None, None, None, None, None, None, None, None, None, None, None) == 1
    assert lib.mpt_enumerate(None, None, None, 2, None, None, None, None) == 1
    assert lib.mpt_ctx_destroy(None) == 1
    assert lib.mpt_ctx_time_solver(None, 1) == 1
    ms = C.c_float()
    assert lib.mpt_ctx_solver_ms(None, 2, C.byref(ms)) == 1


def _prototypes():
    """name -> (return type, [argument types]) parsed from include/mpt.h."""
    text = open(os.path.join(ROOT, "include", "mpt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for ret, name, args in re.findall(r"([A-Za-z_][\w \*]*?)\s*\b(mpt_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text):
        parts = [a.strip() for a in args.replace("\n", " ").split(",") if a.strip() and a.strip() != "void"]
        # drop the parameter name, keep the type (with any '*')
        types = [re.sub(r"\b[A-Za-z_]\w*\s*$", "", a).strip() if not a.endswith("*") else a for a in parts]
        out[name] = (ret.strip(), types)
    return out


def _kind_c(t: str) -> str:
    if "*" in t:
        return "ptr"
    t = t.replace("const", "").strip()
    return {"int": "i32", "int32_t": "i32", "int64_t": "i64", "uint64_t": "u64", "double": "f64",
            "float": "f32"}[t]


def _kind_ctypes(t) -> str:
    if t in (C.c_void_p, C.c_char_p) or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "ptr"
    for k, ct in (("i32", C.c_int32), ("i64", C.c_int64), ("u64", C.c_uint64), ("f64", C.c_double),
                  ("f32", C.c_float)):
        if t is ct:
            return k
    raise AssertionError(t)


def test_binding_signatures_match_the_header(lib):
    protos = _prototypes()
    from paper_2301_06399_gb300 import mpt

    assert sorted(protos) == sorted(mpt.SYMBOLS)
    for name, (ret, args) in protos.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == len(args), (name, len(fn.argtypes), args)
        for i, (want, got) in enumerate(zip(args, fn.argtypes)):
            assert _kind_c(want) == _kind_ctypes(got), (name, i, want, got)
        want_ret = _kind_c(ret)
        got_ret = "i32" if fn.restype is C.c_int else _kind_ctypes(fn.restype)
        assert want_ret == got_ret, (name, ret, fn.restype)
