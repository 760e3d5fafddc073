"""The C ABI library loads and exports every function include/mapper.h
declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    text = open(os.path.join(ROOT, "include", "mapper.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(mapper_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2011_03209_gb300 import _capi, build
    build.build()
    return _capi.load()


def test_header_lists_the_api():
    names = _declared()
    for must in ("mapper_lens", "mapper_cover", "mapper_cluster", "mapper_nerve", "mapper_graph"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2011_03209_gb300 import _capi
    names = _declared()
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(_capi.EXPORTS)


def test_abi_version_and_strings(lib):
    assert lib.mapper_abi_version() == 6
    assert lib.mapper_strerror(0) == b"ok"
    assert lib.mapper_strerror(-4) == b"device wait timed out"


def test_struct_layouts_match_header():
    from paper_2011_03209_gb300 import _capi
    # mapper_params: 7 int32, pad to 8, 2 doubles, double, 3 int32, pad to 8, 2 doubles
    assert ctypes.sizeof(_capi.MapperParams) == 88
    assert _capi.MapperParams.overlap.offset == 32
    assert _capi.MapperParams.cover_kind.offset == 64
    assert _capi.MapperParams.lens_param.offset == 72
    assert ctypes.sizeof(_capi.MapperStats) == 8 * 41


def test_null_and_bad_arguments_are_rejected_without_a_gpu(lib):
    from paper_2011_03209_gb300 import _capi
    assert lib.mapper_graph(None, None, 0, 0, 0, None, None) == _capi.MAPPER_EINVAL
    assert lib.mapper_cover_sizes(None, None, None) == _capi.MAPPER_EINVAL
    assert lib.mapper_stats_get(None, None) == _capi.MAPPER_EINVAL
    lib.mapper_free(None)
    assert lib.mapper_last_error()


def test_knobs_and_new_calls_reject_a_null_context_without_a_gpu(lib):
    """The tuning knobs, the failure self-test and the extended lens call
    validate their context before touching a device."""
    from paper_2011_03209_gb300 import _capi
    assert lib.mapper_set_pass1_tile_n(None, 0) == _capi.MAPPER_EINVAL
    assert lib.mapper_set_cross_screen(None, 0) == _capi.MAPPER_EINVAL
    assert lib.mapper_set_knn_screen(None, 0) == _capi.MAPPER_EINVAL
    assert lib.mapper_set_band_queue_cap(None, 0) == _capi.MAPPER_EINVAL
    assert lib.mapper_set_pass1_screen(None, 0) == _capi.MAPPER_EINVAL
    assert lib.mapper_single_linkage(None, None, 0, 0, 0, None, 1.0, None) == _capi.MAPPER_EINVAL
    assert lib.mapper_forest_sizes(None, None) == _capi.MAPPER_EINVAL
    assert lib.mapper_forest_cut(None, None, 1.0, None) == _capi.MAPPER_EINVAL
    assert lib.mapper_selftest_mma_error(None, 64, 1, 0, 1, None, None) == _capi.MAPPER_EINVAL
    assert lib.mapper_selftest_wait(None) == _capi.MAPPER_EINVAL
    assert lib.mapper_lens_ex(None, None, 0, 0, 0, 1, None, None, None, 1, None, None) == _capi.MAPPER_EINVAL
    assert lib.mapper_knn_distance(None, None, 0, 0, 0, None, 0, 1, None) == _capi.MAPPER_EINVAL
    assert lib.mapper_set_timing(None, 1) == _capi.MAPPER_EINVAL


def test_footprint_counts_a_density_lens_without_a_gpu(lib):
    """The footprint of a graph with a density filter covers the one-element
    clustering of the whole cloud that computes it."""
    import ctypes
    from paper_2011_03209_gb300 import _capi
    import paper_2011_03209_gb300 as mg
    n, d = 1_000_000, 256
    l2 = mg.params((mg.LENS_L2,), (0,), (100,), (0.2,), 20.0, 5, mg.BF16)
    den = mg.params((mg.LENS_DENSITY,), (0,), (100,), (0.2,), 20.0, 5, mg.BF16, lens_param=(20.0,))
    b_l2, b_den = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.mapper_graph_footprint(n, d, ctypes.byref(l2), ctypes.byref(b_l2)) == _capi.MAPPER_OK
    assert lib.mapper_graph_footprint(n, d, ctypes.byref(den), ctypes.byref(b_den)) == _capi.MAPPER_OK
    assert b_den.value >= b_l2.value > n * d * 4


def test_header_compiles_as_c_and_links(lib, tmp_path):
    """A plain C99 program includes include/mapper.h, links the library and
    calls it without a GPU (version, error strings, argument checks): the
    boundary is C, not C++."""
    import shutil
    import subprocess
    from paper_2011_03209_gb300 import _capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_abi.c"
    src.write_text(r"""
#include <stdio.h>
#include "mapper.h"
int main(void) {
    mapper_stats st;
    size_t bytes = 0;
    mapper_params p = {0};
    if (mapper_abi_version() != MAPPER_ABI_VERSION) return 1;
    if (mapper_graph(NULL, NULL, 0, 0, 0, NULL, NULL) != MAPPER_EINVAL) return 2;
    if (mapper_stats_get(NULL, &st) != MAPPER_EINVAL) return 3;
    p.m = 1; p.lens_kind[0] = MAPPER_LENS_L2; p.n_intervals[0] = 10; p.overlap[0] = 0.25;
    p.eps = 1.0; p.min_pts = 5; p.precision = MAPPER_BF16; p.cover_kind = MAPPER_COVER_UNIFORM;
    if (mapper_graph_footprint(1000, 16, &p, &bytes) != MAPPER_OK || bytes == 0) return 4;
    printf("%s|%s|%zu|%zu\n", mapper_strerror(MAPPER_OK), mapper_strerror(MAPPER_ETIMEOUT),
           sizeof(mapper_stats), sizeof(mapper_params));
    return 0;
}
""")
    exe = tmp_path / "use_abi"
    libdir = os.path.dirname(_capi.LIB_PATH)
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), "-L", libdir, "-lmapper_gb300", "-Wl,-rpath," + libdir],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    ok, timeout, n_stats, n_params = out.stdout.strip().split("|")
    assert (ok, timeout) == ("ok", "device wait timed out")
    # the ctypes mirrors of the structs have the C layout's sizes
    assert int(n_stats) == ctypes.sizeof(_capi.MapperStats)
    assert int(n_params) == ctypes.sizeof(_capi.MapperParams)


def test_checked_build_exports_every_symbol():
    """The checked build (device-side index checks turning an out-of-range
    index into MAPPER_EINTERNAL) builds from the same sources and exports the
    same C ABI."""
    from paper_2011_03209_gb300 import _capi, build
    path = build.build(checked=True)
    lib = ctypes.CDLL(path)
    for name in _capi.EXPORTS:
        assert hasattr(lib, name), name
    lib.mapper_abi_version.restype = ctypes.c_int
    assert lib.mapper_abi_version() == 6
