"""Host-side checks of the C ABI (no GPU needed): the library loads and exports
every entry point include/rankest.h declares, and the binding knows them all."""
import ctypes
import os
import re

import pytest

from paper_2105_07388_gb300 import build, rankest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(re_\w+)\s*\(", text, flags=re.M):
            names.add(mt.group(1))
    return names


@pytest.fixture(scope="module")
def built():
    return build.build()


def test_header_and_binding_agree():
    assert declared_functions() == set(rankest.EXPORTED)


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built)
    for name in declared_functions():
        assert hasattr(L, name), name


def test_version_and_defaults(built):
    assert rankest.re_version() >= 100
    o = rankest.re_opts_default()
    assert (o.s0, o.s_max, o.precision, o.y_kind) == (8, 512, rankest.RE_PREC_FP32, -1)


def test_create_without_gpu_fails_cleanly(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rankest.RankEstError) as ei:
        rankest.re_create(0)
    assert ei.value.code in (rankest.RE_ERR_CUDA, rankest.RE_ERR_ARG)


def _header_layout(tmp_path):
    """Sizes and field offsets of the header's structs and the values of its
    RE_* constants, as a C compiler sees them (gcc on this host)."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    structs = {name: [f for f, _ in getattr(rankest, name)._fields_]
               for name in ("re_opts", "re_result", "re_block", "re_kblock", "re_stats", "re_qb_result")}
    consts = [n for n in dir(rankest) if re.fullmatch(r"RE_[A-Z0-9_]+", n)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rankest.h"', "int main(void) {"]
    for s, fields in structs.items():
        lines.append(f'printf("{s} size %zu\\n", sizeof({s}));')
        for f in fields:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    for c in consts:
        lines.append(f'printf("{c} %lld\\n", (long long)({c}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        k, v = ln.rsplit(" ", 1)
        got[k] = int(v)
    return structs, consts, got


def test_binding_layout_matches_header(tmp_path):
    structs, consts, c = _header_layout(tmp_path)
    for s, fields in structs.items():
        cls = getattr(rankest, s)
        assert ctypes.sizeof(cls) == c[f"{s} size"], s
        for f in fields:
            assert getattr(cls, f).offset == c[f"{s}.{f}"], (s, f)
    for name in consts:
        assert getattr(rankest, name) == c[name], name


def test_noalloc_binding_rejects_wrong_dtypes_and_devices():
    """The allocation-free binding checks dtypes and devices before any C call
    (CPU tensors are never passed to the library)."""
    import torch
    A = torch.zeros(64, 32)
    with pytest.raises(ValueError, match="float32"):
        rankest.re_sketch_apply_noalloc(A, 0, 8, 1, torch.zeros(64, 8, dtype=torch.float64))
    with pytest.raises(ValueError, match="float64"):
        rankest.re_sketch_apply_noalloc(A, 0, 8, 1, torch.zeros(64, 8), torch.zeros(16, 8))
    with pytest.raises(ValueError, match="CUDA"):
        rankest.re_sketch_apply_noalloc(A, 0, 8, 1, torch.zeros(64, 8), torch.zeros(16, 8, dtype=torch.float64))
