"""CPU-side checks of the CUDA library: it loads, exports every entry point
declared in include/gavis.h, and its host-only helpers are correct.  No kernel
is launched here."""
import ctypes as C
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2605_30342_gb300 as gv
    return gv.load()


def declared():
    src = open(os.path.join(ROOT, "include", "gavis.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gavis_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 10
    for nm in names:
        assert hasattr(lib, nm), nm


def test_binding_exports_match_header():
    import paper_2605_30342_gb300 as gv
    assert set(gv.EXPORTS) <= set(declared())


def test_params_default_are_the_paper_defaults(lib):
    import paper_2605_30342_gb300 as gv
    p = gv.Params()
    assert (p.kappa, p.vf_degree, p.eps_T, p.q_cut, p.beta, p.o0) == (1.0, 2, pytest.approx(1e-4), 9.0, 0.5,
                                                                      pytest.approx(0.15))
    assert p.sigma_c2 == pytest.approx(0.01) and p.logdet_Q0 == 0.0 and p.tile == 16
    assert p.views_per_batch == 0 and p.tile_lists == 0


def test_host_vmf_coefficients_match_oracle(lib):
    import oracle
    import paper_2605_30342_gb300 as gv
    for L in (3, 5):
        for kappa in (0.0, 0.1, 0.3, 0.5, 1.0, 3.0, 4.5, 10.0):
            a = gv.Context.vmf_coeffs(L, kappa)
            b = oracle.vmf_coeffs(L, kappa)
            for l in range(L + 1):
                assert a[l] == pytest.approx(b[l], rel=1e-9, abs=1e-15), (L, kappa, l)
    assert gv.Context.vmf_coeffs(0, 0.0)[0] == pytest.approx(4 * math.pi)


def test_bad_arguments_rejected_without_gpu(lib):
    import paper_2605_30342_gb300 as gv
    assert lib.gavis_vmf_coeffs(6, 1.0, (C.c_double * 7)()) == gv.ERR_ARG
    assert lib.gavis_vmf_coeffs(2, -1.0, (C.c_double * 3)()) == gv.ERR_ARG
    assert lib.gavis_params_default(None) == gv.ERR_ARG


def test_context_creation_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2605_30342_gb300 as gv
    with pytest.raises(gv.GavisError):
        gv.Context(0)
