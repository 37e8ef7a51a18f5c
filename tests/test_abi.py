"""The C ABI library loads and exports every entry point ``include/psc.h``
declares; host-only calls (sizes, validation) work without a GPU."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "psc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(psc_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2012_04838_gb300 import binding, build
    if not os.path.exists(binding.lib_path()):
        build.build()
    return binding.load()


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("psc_workspace_size", "psc_create", "psc_init_field", "psc_step",
              "psc_spectra_and_stats", "psc_rhs", "psc_get_state", "psc_set_state", "psc_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2012_04838_gb300 import binding
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    bound = {n for n, _, _ in binding.EXPORTS}
    assert set(_declared()) <= bound


def test_struct_layouts_match_header(lib, tmp_path):
    import shutil
    import subprocess
    from paper_2012_04838_gb300.binding import CParams, CStats
    # psc_params: 10 int32 + 9 double + 1 uint64 = 120 bytes; psc_stats: 36 doubles + int64
    assert ct.sizeof(CParams) == 120
    assert ct.sizeof(CStats) == 37 * 8
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler to cross-check the header layout")
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "psc.h"\n'
                   'int main(){printf("%zu %zu\\n", sizeof(psc_params), sizeof(psc_stats));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call([cc, "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    a, b = map(int, subprocess.check_output([str(exe)]).split())
    assert (a, b) == (ct.sizeof(CParams), ct.sizeof(CStats))


def test_supported_sizes_and_validation(lib):
    from paper_2012_04838_gb300 import binding as B
    sizes = B.supported_sizes()
    for n in (32, 64, 96, 128, 192, 256, 512, 520, 1024):
        assert n in sizes
    p = B.Params(N=32)
    assert B.workspace_size(p) > 0
    # workspace grows like N^3 and doubles with FP64
    w64 = B.workspace_size(B.Params(N=64, precision=B.FP64))
    w64f = B.workspace_size(B.Params(N=64, precision=B.FP32_MIXED))
    assert 1.8 < w64 / w64f < 2.1
    with pytest.raises(B.PscError) as e:
        B.workspace_size(B.Params(N=100))
    assert e.value.status == B.PSC_EUNSUPPORTED_N
    with pytest.raises(B.PscError) as e:
        B.workspace_size(B.Params(N=32, Sc=0.0))
    assert e.value.status == B.PSC_EINVAL
    with pytest.raises(B.PscError):
        B.workspace_size(B.Params(N=32, dt=0.0, cfl=0.0))


def test_workspace_at_full_size_fits_one_gpu(lib):
    from paper_2012_04838_gb300 import binding as B
    w = B.workspace_size(B.Params(N=1024, precision=B.FP32_MIXED))
    assert 40e9 < w < 80e9
    w = B.workspace_size(B.Params(N=512, precision=B.FP64))
    assert w < 40e9


def test_dealiasing_and_form_validation(lib):
    """Host-side checks of the dealiasing option and of the forms each grid has."""
    from paper_2012_04838_gb300 import binding as B
    PS = B.DEALIAS_PHASE_SHIFT
    for n in (16, 256, 512, 520, 1024):
        w2 = B.workspace_size(B.Params(N=n, precision=B.FP32_MIXED))
        wp = B.workspace_size(B.Params(N=n, precision=B.FP32_MIXED, dealias=PS))
        # the sphere's cube is (sqrt(2) N / 3)^3 / (N / 3)^3 ~ 2.8 times the 2/3 cube's,
        # plus the products of the unshifted grid
        assert 1.8 < wp / w2 < 3.6, (n, wp / w2)
    with pytest.raises(B.PscError) as e:
        B.workspace_size(B.Params(N=32, dealias=2))
    assert e.value.status == B.PSC_EINVAL
    cp = B.Params(N=32).c()
    cp.reserved = 1
    import ctypes as ct
    n = ct.c_size_t()
    assert lib.psc_workspace_size(ct.byref(cp), ct.byref(n)) == B.PSC_EINVAL
    # the convective form exists wherever a register X pass does
    for n, dl in ((256, PS), (512, PS), (1024, PS), (512, B.DEALIAS_TWO_THIRDS)):
        assert B.workspace_size(B.Params(N=n, precision=B.FP32_MIXED, dealias=dl,
                                         nonlinear_form=B.NL_CONVECTIVE)) > 0
    # ... and not at 520, whose rows only have the shared-memory row X pass
    for dl in (B.DEALIAS_TWO_THIRDS, PS):
        with pytest.raises(B.PscError) as e:
            B.workspace_size(B.Params(N=520, precision=B.FP32_MIXED, dealias=dl,
                                      nonlinear_form=B.NL_CONVECTIVE))
        assert e.value.status == B.PSC_EUNSUPPORTED_N
    # compact shapes follow the retained half-width
    assert B.compact_shape(520) == (4, 347, 347, 174)
    assert B.compact_shape(520, PS) == (4, 491, 491, 246)
    # the sphere's cube at 1024^3: half-width 482 (9 k^2 < 2 N^2) widened to 483
    # so that a kx row holds an even number of values (TMA-staged passes)
    assert B.compact_shape(1024, PS) == (4, 967, 967, 484)
    assert B.compact_shape(256, PS) == (4, 243, 243, 122)
    assert B.compact_shape(512, PS) == (4, 483, 483, 242)
