"""Host-side bounds check of the split path's index tables (favest_debug_check_layout; no
GPU): for a sweep of degrees, batches, field types and tile widths, every tensor-core GEMM
work item's operand chunks and TMA box coordinates (the Legendre operand's row blocks and
latitude blocks, the coefficient and field operands) and its output rows stay inside the
buffers they address and inside the rows of their own order, and the per-(order, parity)
regions are in range, aligned and disjoint.  Degrees: every L up to 160 (the small-tile,
padding and equator cases), both sides of the latitude-tile boundaries (J = 128, 256, 384,
512), the paper's timing degrees (Table 3) up to L = 1250, and L = 2047.  The check's own
sensitivity is shown by corrupting its copy of the tables (poison modes), which it must
report."""
import pytest

from paper_1908_00041_gb300 import api

C64, R32 = api.FAVEST_IO_C64, api.FAVEST_IO_R32


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00041_gb300 import build
    build.build()
    return api.lib()


def _ok(L, B, io, gemm_n=0):
    st, msg = api.debug_check_layout(L, B, api.FAVEST_BF16X6, io, gemm_n)
    assert st == api.FAVEST_OK, (L, B, io, gemm_n, st, msg)


def test_all_small_degrees(lib):
    for L in range(1, 161):
        for B in (1, 2, 3, 17):
            _ok(L, B, C64)
        _ok(L, 5, R32)
        _ok(L, 2, C64, 256)


@pytest.mark.parametrize("L", [253, 254, 255, 256, 511, 512, 765, 766, 767, 768, 1023, 1024])
def test_tile_boundaries(lib, L):
    for B, io, gn in ((1, C64, 0), (16, C64, 0), (17, C64, 0), (32, C64, 0), (33, C64, 0), (64, R32, 0),
                      (3, C64, 256)):
        _ok(L, B, io, gn)


@pytest.mark.parametrize("L", [250, 500, 750, 1000, 1250, 2047])
def test_timing_degrees(lib, L):
    _ok(L, 32 if L <= 1250 else 8, C64)
    _ok(L, 7, R32)


def test_fp64_plans_have_no_tables(lib):
    assert api.debug_check_layout(1023, 32, api.FAVEST_FP64, api.FAVEST_IO_C128)[0] == api.FAVEST_OK


def test_arguments_as_plan_create(lib):
    assert api.debug_check_layout(0, 1)[0] == api.FAVEST_EINVAL
    assert api.debug_check_layout(16, 0)[0] == api.FAVEST_EINVAL
    assert api.debug_check_layout(2560, 1)[0] == api.FAVEST_EUNSUPPORTED
    assert api.debug_check_layout(16, 1, api.FAVEST_BF16X6, api.FAVEST_IO_C128)[0] == api.FAVEST_EUNSUPPORTED
    assert api.debug_check_layout(16, 1, gemm_n=128)[0] == api.FAVEST_EINVAL
    assert api.debug_check_layout(16, 1, poison=4)[0] == api.FAVEST_EINVAL


@pytest.mark.parametrize("poison,what", [(1, "forward item B box"), (2, "adjoint item"),
                                         (3, "Legendre row blocks")])
def test_check_reports_corrupted_tables(lib, poison, what):
    for L, B in ((16, 2), (255, 8), (1023, 32)):
        st, msg = api.debug_check_layout(L, B, poison=poison)
        assert st == api.FAVEST_EINTERNAL, (L, B, poison, st)
        assert msg.startswith(what), msg
