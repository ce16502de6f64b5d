"""The C-ABI library loads and exports every symbol ``include/vi.h`` declares.

No compute call is made here (no GPU is needed): only host-side argument
checks that return before any CUDA work.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_06134_gb300 import build, vi
    build.build()
    return vi.library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "vi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vi_[a-z_]+)\s*\(", text)))


def test_header_declares_the_paper_boundary():
    names = declared_functions()
    for required in ("vi_load_volume", "vi_set_transfer_function", "vi_set_light",
                     "vi_build_attenuation", "vi_render"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2008_06134_gb300 import vi
    names = declared_functions()
    assert sorted(vi.EXPORTS) == names
    for name in names:
        assert hasattr(lib, name), name


def test_error_strings(lib):
    from paper_2008_06134_gb300 import vi
    for code in (vi.OK, vi.EINVAL, vi.ENOMEM, vi.ESTATE, vi.ECUDA, vi.ETIMEOUT):
        assert vi.error_string(code) and vi.error_string(code) != "unknown status"
    assert vi.error_string(12345) == "unknown status"


def test_null_context_is_rejected_without_cuda(lib):
    from paper_2008_06134_gb300 import vi
    null = C.c_void_p(None)
    f3 = (C.c_float * 3)(0, 0, 1)
    assert lib.vi_destroy(null) == vi.EINVAL
    assert lib.vi_set_memory_budget(null, 0) == vi.EINVAL
    assert lib.vi_load_volume(null, null, 0, 1, 1, 1, 0) == vi.EINVAL
    assert lib.vi_set_transfer_function(null, null, 2, 0.0, 1.0) == vi.EINVAL
    assert lib.vi_set_light(null, f3, f3) == vi.EINVAL
    assert lib.vi_build_attenuation(null, 1, 1, 0, None) == vi.EINVAL
    assert lib.vi_render(null, None, 1, 1, 0.5, null, 0, None) == vi.EINVAL
    assert lib.vi_sync(null) == vi.EINVAL
    assert lib.vi_attenuation_info(null, None, None, None, None) == vi.EINVAL
    assert lib.vi_get_attenuation(null, null, 0, 0) == vi.EINVAL
    assert lib.vi_launch_count(null, None) == vi.EINVAL
    assert lib.vi_get_skip_grid(null, None, None, 0, None, 0) == vi.EINVAL
    assert lib.vi_create(None, 0, null) == vi.EINVAL


def test_binding_does_not_import_the_oracle():
    src = open(os.path.join(ROOT, "paper_2008_06134_gb300", "vi.py")).read()
    assert "oracle" not in re.sub(r'""".*?"""', "", src, flags=re.S)
    for f in os.listdir(os.path.join(ROOT, "paper_2008_06134_gb300", "csrc")):
        assert "oracle" not in open(os.path.join(ROOT, "paper_2008_06134_gb300", "csrc", f)).read()


def test_server_calls_reject_bad_arguments_without_cuda(lib):
    from paper_2008_06134_gb300 import vi
    null = C.c_void_p(None)
    st, res = C.c_int(), C.c_int()
    assert lib.vi_server_destroy(null) == vi.EINVAL
    assert lib.vi_server_submit(null, None, None) == vi.EINVAL
    assert lib.vi_server_wait(null, 1, 0.0, C.byref(st), C.byref(res)) == vi.EINVAL
    assert lib.vi_server_cancel(null, 1) == vi.EINVAL
    assert lib.vi_server_get_stats(null, None) == vi.EINVAL
    assert lib.vi_server_set_graphs(null, 1) == vi.EINVAL
    assert lib.vi_server_set_eviction(null, vi.EVICT_COST) == vi.EINVAL
    assert lib.vi_server_create(None, 0, 4, 0, 0) == vi.EINVAL
    h = C.c_void_p()
    assert lib.vi_server_create(C.byref(h), 0, 0, 0, 0) == vi.EINVAL      # no slots
    rc = lib.vi_server_create(C.byref(h), 0, 2, 0, 0)
    if rc == vi.OK:          # a GPU is present: clean up
        assert lib.vi_server_destroy(h) == vi.OK
    else:                    # no GPU here: a clean error, no crash
        assert rc in (vi.ECUDA, vi.EINVAL)


def test_checked_library_exports_every_symbol_and_reports_its_kind(lib):
    """libvi_checked.so (VI_DEBUG_BOUNDS=1) exports the same ABI; the release
    library answers vi_debug_bounds with VI_ESTATE without touching CUDA."""
    from paper_2008_06134_gb300 import vi
    checked = vi.library(checked=True)
    for name in declared_functions():
        assert hasattr(checked, name), name
    n, site, idx = C.c_uint64(7), C.c_int(7), C.c_int64(7)
    for L in (lib, checked):
        assert L.vi_debug_bounds(0, None, None, None) == vi.EINVAL
    assert lib.vi_debug_bounds(0, C.byref(n), C.byref(site), C.byref(idx)) == vi.ESTATE
    assert (n.value, site.value, idx.value) == (0, 0, 0)
