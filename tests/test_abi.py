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
