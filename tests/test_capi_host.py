"""Host-side checks of the C ABI (no GPU): the library builds and loads, exports
every entry point declared in include/gbs.h, rejects invalid problem
descriptions before touching the GPU, and sizes states/workspaces correctly.
Also cross-checks the product's scheme table against the paper's printed values
(tests/golden/paper_schemes.txt)."""
import ctypes
import os
import re
from fractions import Fraction

import pytest

from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import build as Bld
from paper_1907_11771_gb300 import schemes as S
from tests.conftest import ROOT, load_golden


@pytest.fixture(scope="module")
def libpath():
    return Bld.build()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbs_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    syms = declared_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(L, s), s
    # the binding wraps every declared entry point under the same name
    for s in syms:
        assert hasattr(B, s), s


def test_invalid_problems_rejected_without_gpu(libpath):
    B.lib()
    bad = [
        dict(system=3, ndim=1, fd_order=4),
        dict(system=B.GBS_WAVE1D, ndim=2, fd_order=4),
        dict(system=B.GBS_ACOUSTIC, ndim=2, fd_order=5),
        dict(system=B.GBS_ACOUSTIC, ndim=4, fd_order=4),
    ]
    for kw in bad:
        pb = B.make_problem(kw["system"], kw["ndim"], kw["fd_order"], B.GBS_F64, [(16, 16, 1)], [(1.0, 1.0, 1.0)])
        with pytest.raises(B.GbsError) as e:
            B.gbs_create(pb)
        assert e.value.status == 1
        assert B.gbs_state_elems(pb) == 0
    # a grid smaller than the stencil radius, and a non-unit unused dimension
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 6, B.GBS_F64, [(2, 16, 1)], [(1.0, 1.0, 1.0)])
    with pytest.raises(B.GbsError):
        B.gbs_create(pb)
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 4, B.GBS_F64, [(16, 16, 2)], [(1.0, 1.0, 1.0)])
    with pytest.raises(B.GbsError):
        B.gbs_create(pb)
    # the spectral one-way wave: fd_order 0, FP64, power-of-two sizes up to 2048
    for prec, order, n in ((B.GBS_F64, 4, 64), (B.GBS_F32_STATE_F64_COMBINE, 0, 64), (B.GBS_F64, 0, 48),
                           (B.GBS_F64, 0, 4096)):
        pb = B.make_problem(B.GBS_ONEWAY_SPECTRAL, 1, order, prec, [(n, 1, 1)], [(1.0 / n, 1.0, 1.0)])
        with pytest.raises(B.GbsError):
            B.gbs_create(pb)
    pb = B.make_problem(B.GBS_ONEWAY_SPECTRAL, 1, 0, B.GBS_F64, [(256, 1, 1)], [(1.0 / 256, 1.0, 1.0)])
    assert B.gbs_state_elems(pb) == 256
    # 2^31 grid points in one problem (32-bit point indices inside the kernels)
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 4, B.GBS_F32_STATE_F64_COMBINE, [(65536, 32768, 1)], [(1.0, 1.0, 1.0)])
    with pytest.raises(B.GbsError):
        B.gbs_create(pb)
    assert B.gbs_state_elems(pb) == 0
    # an unknown precision
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 4, 3, [(16, 16, 1)], [(1.0, 1.0, 1.0)])
    with pytest.raises(B.GbsError):
        B.gbs_create(pb)
    assert B.gbs_state_elems(pb) == 0
    # wave system with media is refused before any device call
    pb = B.make_problem(B.GBS_WAVE1D, 1, 4, B.GBS_F64, [(16,)], [(1.0,)])
    with pytest.raises(B.GbsError):
        B.gbs_create(pb, kappa=1234, rho=5678)
    assert "media" in B.gbs_last_error(None)


def test_state_and_workspace_sizes(libpath):
    B.lib()
    pb = B.make_problem(B.GBS_ACOUSTIC, 2, 6, B.GBS_F32_STATE_F64_COMBINE, [(128, 64), (32, 32)], [(1, 1), (1, 1)])
    assert B.gbs_state_elems(pb) == 3 * (128 * 64 + 32 * 32)
    ws = B.gbs_workspace_bytes(pb, 22)
    E = 3 * (128 * 64 + 32 * 32)
    assert ws >= 4 * 4 * E + 8 * E
    pb3 = B.make_problem(B.GBS_ACOUSTIC, 3, 4, B.GBS_F64, [(8, 9, 10)], [(1, 1, 1)], enable_adjoint=True)
    assert B.gbs_state_elems(pb3) == 4 * 8 * 9 * 10
    assert B.gbs_workspace_bytes(pb3, 22) > B.gbs_workspace_bytes(pb3, 2)
    # FP32-pair precision: FP64-sized levels plus pair copies of y_in, kappa and b
    pbx = B.make_problem(B.GBS_ACOUSTIC, 2, 6, B.GBS_F32X2, [(128, 64)], [(1, 1)])
    pbd = B.make_problem(B.GBS_ACOUSTIC, 2, 6, B.GBS_F64, [(128, 64)], [(1, 1)])
    assert B.gbs_workspace_bytes(pbx, 22) == B.gbs_workspace_bytes(pbd, 22) + 8 * (3 + 2) * 128 * 64


def test_product_scheme_table_matches_printed_values():
    gold = load_golden("paper_schemes.txt")
    pairs = [("gbs_8_6", S.GBS_8_6), ("gbs_8_8", S.GBS_8_8), ("gbs_12_8", S.GBS_12_8),
             ("table1_order8", S.SQ8_TABLE1), ("table1_order12", S.SQ12_TABLE1), ("table1_order16", S.SQ16_TABLE1)]
    for key, sc in pairs:
        g = gold[key]
        assert sc.order == int(g["order"])
        assert list(sc.steps_dep) == [int(t) for t in g["dep"].split()]
        assert list(sc.steps_free) == [int(t) for t in g.get("free", "").split()]
        assert [Fraction(t) for t in sc.c_free_text] == [Fraction(t) for t in g.get("cfree", "").split()]
        assert sc.evals_per_core == int(g["evals"])
    assert S.GBS_8_6.updates_per_point == 143
    assert S.GBS_8_8.updates_per_point == 255
    assert S.SQ8_2468.updates_per_point == 24


def test_entry_points_refuse_a_null_handle_without_gpu(libpath):
    # every stepping call checks its handle before any device work, the host-stream call
    # included (its arrays of host buffers are checked next)
    L = B.lib()
    ptrs = (ctypes.c_void_p * 1)(None)
    assert L.gbs_step_host_stream(None, ptrs, ptrs, 1, ctypes.c_double(0.1), 1) == 1
    assert L.gbs_step_host(None, None, None, ctypes.c_double(0.1), 1) == 1
    assert L.gbs_step(None, None, None, ctypes.c_double(0.1), 1) == 1
    assert L.gbs_set_option(None, b"tma", 1) == 1


def test_noalloc_refuses_invalid_descriptions_without_gpu(libpath):
    # the allocation-free entry point checks the description, the media and the state pointers
    # before its first device call, and leaves a message naming the problem
    B.lib()
    sq = S.SQ8_2468
    args = (sq.order, sq.steps_dep, sq.steps_free, [])
    cases = [
        (B.make_problem(3, 1, 4, B.GBS_F64, [(16,)], [(1.0,)]), None, None, 1, 1, "system"),
        (B.make_problem(B.GBS_WAVE1D, 2, 4, B.GBS_F64, [(16, 16)], [(1.0, 1.0)]), None, None, 1, 1, "ndim"),
        (B.make_problem(B.GBS_ACOUSTIC, 2, 5, B.GBS_F64, [(16, 16)], [(1.0, 1.0)]), 1, 1, 1, 1, "fd_order"),
        (B.make_problem(B.GBS_ACOUSTIC, 2, 4, B.GBS_F32X2, [(16, 16)], [(1.0, 1.0)]), 1, 1, 1, 1, "precision"),
        (B.make_problem(B.GBS_ACOUSTIC, 2, 4, B.GBS_F64, [(16, 16)], [(1.0, 1.0)], enable_adjoint=True),
         1, 1, 1, 1, "adjoint"),
        (B.make_problem(B.GBS_ACOUSTIC, 2, 4, B.GBS_F64, [(16, 16)], [(1.0, 1.0)]), None, None, 1, 1, "kappa"),
        (B.make_problem(B.GBS_WAVE1D, 1, 4, B.GBS_F64, [(16,)], [(1.0,)]), 1, 1, 1, 1, "kappa"),
        (B.make_problem(B.GBS_WAVE1D, 1, 4, B.GBS_F64, [(16,)], [(1.0,)]), None, None, None, 1, "NULL"),
    ]
    for pb, kappa, rho, y_in, y_out, word in cases:
        with pytest.raises(B.GbsError) as e:
            B.gbs_step_noalloc(pb, kappa, rho, *args, y_in, y_out, 0.1, 1)
        assert e.value.status == 1
        assert word in B.gbs_noalloc_last_error(), (word, B.gbs_noalloc_last_error())
    assert B.lib().gbs_step_noalloc(None, None, None, 8, 4, None, 0, None, None, None, None,
                                    ctypes.c_double(0.1), 1, None) == 1
    assert "NULL" in B.gbs_noalloc_last_error()


def test_every_declaration_cites_its_passage_or_says_it_has_none():
    # each entry point's comment names the section, equation or appendix that defines the
    # operation, or states that the paper has no counterpart
    src = open(os.path.join(ROOT, "include", "gbs.h")).read()
    cite = re.compile(r"Sec\. \d|App\. [AB]|eq\. \"|no counterpart|not in the paper", re.I)
    names = []
    for m in re.finditer(r"^[a-z][a-z_0-9 *]*\b(gbs_[a-z_0-9]+)\s*\(", src, flags=re.M):
        before = src[:m.start()]
        comment = before[before.rfind("/*"):before.rfind("*/")]
        comment = re.sub(r"\s*\n\s*\*\s*", " ", comment)
        assert cite.search(comment), m.group(1)
        names.append(m.group(1))
    assert set(names) == set(declared_symbols())
