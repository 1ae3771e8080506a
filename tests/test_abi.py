"""The C-ABI library loads, exports every symbol include/egm.h declares, and its
struct layouts match the Python binding.  No compute calls (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "egm.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g

    g.build()
    from paper_2603_18401_gb300 import _egm

    return _egm.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(egm_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("egm_create", "egm_destroy", "egm_match_pair", "egm_match_batch", "egm_intervals",
              "egm_match_pair_host", "egm_sync", "egm_status_string"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2603_18401_gb300 import _egm

    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_egm.SIGNATURES), "binding and header disagree"
    out = subprocess.run(["nm", "-D", "--defined-only", _egm.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (egm_\w+)", out))
    assert set(names) <= exported


def test_struct_layouts_match_c(tmp_path):
    from paper_2603_18401_gb300 import _egm

    src = tmp_path / "layout.c"
    fields = {"egm_pair": _egm.egm_pair, "egm_out": _egm.egm_out, "egm_params": _egm.egm_params,
              "egm_stats": _egm.egm_stats, "egm_timing": _egm.egm_timing}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "egm.h"', "int main(void){"]
    for s, cls in fields.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for s, cls in fields.items():
        assert int(got[s]) == C.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def test_status_strings_and_version(lib):
    assert lib.egm_version() == 1
    for s in range(-8, 1):
        assert lib.egm_status_string(s)
    p = __import__("paper_2603_18401_gb300")._egm.egm_params()
    lib.egm_default_params(C.byref(p))
    assert (p.ratio_num, p.ratio_den, p.sync) == (4, 5, 1)


def test_create_without_gpu_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = C.c_void_p()
    assert lib.egm_create(C.byref(ctx), 0, None) == -2  # EGM_ERR_CUDA
    assert not ctx.value
    assert lib.egm_destroy(None) == 0
    assert lib.egm_match_pair(None, None, None) == -1   # EGM_ERR_ARG


def test_matcher_requires_library_and_gpu():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2603_18401_gb300 import Matcher

    with pytest.raises(Exception):
        Matcher(0)


def test_header_constants_match_binding():
    """Every #define and enum value of the header has the same value in the binding."""
    from paper_2603_18401_gb300 import _egm

    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = {k: int(v, 0) for k, v in re.findall(r"#define\s+(EGM_\w+)\s+(-?(?:0x[0-9a-fA-F]+|\d+))\b", text)}
    consts.update({k: int(v) for k, v in re.findall(r"\b(EGM_\w+)\s*=\s*(-?\d+)", text)})
    assert "EGM_MLP_PARAMS" in consts
    for k, v in consts.items():
        if hasattr(_egm, k):
            assert getattr(_egm, k) == v, k
    import synth

    assert consts["EGM_MLP_PARAMS"] == synth.mlp_param_count()
