"""The C ABI without a GPU: the library builds, loads, exports every entry
point declared in include/feti.h, and fails cleanly (status, no abort) when
no CUDA device is present."""
import os
import re

import pytest

import paper_2111_11728_gb300 as fg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "feti.h")).read()
    return sorted(set(re.findall(r"^\s*(?:feti_status|void|const char\*)\s+(feti_\w+)\s*\(", text, re.M)))


def test_header_declares_the_binding_exports():
    assert declared_symbols() == sorted(fg.EXPORTS)


def test_library_exports_every_declared_symbol():
    if not os.path.exists(fg.LIB_PATH):
        from paper_2111_11728_gb300 import build
        build.build()
    L = fg.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_defaults_and_invalid_options():
    o = fg.feti_options_default()
    assert (o.method, o.scaling, o.krylov, o.precision) == (fg.FETI_FETIDP, fg.FETI_SCALING_K, fg.FETI_RRS,
                                                             fg.FETI_FP64)
    assert o.tol == 1e-6 and o.rr_tol == 1e-10 and o.max_iter == 500
    bad = fg.feti_options_default()
    bad.method = 7
    with pytest.raises(fg.FetiError) as e:
        fg.feti_create(bad)
    assert e.value.status == fg.FETI_EINVAL
    assert fg.lib().feti_options_default(None) == fg.FETI_EINVAL


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fg.FetiError) as e:
        fg.feti_create(fg.feti_options_default())
    assert e.value.status == fg.FETI_ECUDA
