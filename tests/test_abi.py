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
    assert fg.lib().feti_set_allocator(None, None) == fg.FETI_EINVAL


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fg.FetiError) as e:
        fg.feti_create(fg.feti_options_default())
    assert e.value.status == fg.FETI_ECUDA


def test_option_combinations_rejected_before_any_device_call():
    o = fg.feti_options_default()
    assert o.primal == fg.FETI_PRIMAL_CORNERS and o.precond == fg.FETI_PRECOND_DIRICHLET
    cases = []
    a = fg.feti_options_default()
    a.primal = 3                                        # no such primal set
    cases.append((a, fg.FETI_EINVAL))
    a2 = fg.feti_options_default()
    a2.primal, a2.primal_jump = fg.FETI_PRIMAL_ADAPTIVE, 0.5   # a jump ratio below 1 selects nothing sensible
    cases.append((a2, fg.FETI_EINVAL))
    a3 = fg.feti_options_default()
    a3.primal, a3.method = fg.FETI_PRIMAL_ADAPTIVE, fg.FETI_TFETI
    cases.append((a3, fg.FETI_EINVAL))
    b = fg.feti_options_default()
    b.primal, b.method = fg.FETI_PRIMAL_EDGES, fg.FETI_TFETI   # primal sets are a FETI-DP choice
    cases.append((b, fg.FETI_EINVAL))
    c = fg.feti_options_default()
    c.primal, c.precond = fg.FETI_PRIMAL_EDGES, fg.FETI_PRECOND_LUMPED
    cases.append((c, fg.FETI_ENOTSUP))
    d = fg.feti_options_default()
    d.precision = 5
    cases.append((d, fg.FETI_EINVAL))
    assert o.refine == fg.FETI_REFINE_DUAL
    e_ = fg.feti_options_default()
    e_.refine = 2                                       # no such refinement residual
    cases.append((e_, fg.FETI_EINVAL))
    for opt, status in cases:
        with pytest.raises(fg.FetiError) as e:
            fg.feti_create(opt)
        assert e.value.status == status


def test_binding_constants_match_the_header():
    """Enumerations of include/feti.h and the binding's constants agree (name and value)."""
    text = open(os.path.join(ROOT, "include", "feti.h")).read()
    values = {name: int(v) for name, v in re.findall(r"\b(FETI_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    checked = 0
    for name, v in values.items():
        if hasattr(fg, name):
            assert getattr(fg, name) == v, name
            checked += 1
    assert checked >= 40
    phases = sorted((v, n) for n, v in values.items() if n.startswith("FETI_PHASE_"))
    assert [n[len("FETI_PHASE_"):].lower() for _, n in phases] == list(fg.PHASES)
    assert values["FETI_N_PHASES"] == len(fg.PHASES)
