"""The C ABI without a GPU: the library loads, exports every function that
include/khop.h declares (and the binding mirrors the same names), and its
argument checks answer before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "khop.h")


@pytest.fixture(scope="module")
def kh():
    import paper_1905_01294_gb300 as kh
    kh.build_library()
    kh.lib()
    return kh


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(khop_\w+)\s*\(", src, re.M)))


def test_header_declares_the_expected_entry_points():
    d = declared()
    for name in ("khop_graph_create", "khop_count", "khop_count_mixed", "khop_submit",
                 "khop_poll", "khop_server_create", "khop_server_destroy", "khop_get_error",
                 "khop_count_static", "khop_batch_stats"):
        assert name in d


def test_library_exports_every_declared_function(kh):
    L = kh.lib()
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(kh.EXPORTS) == declared()


def test_status_strings_and_version(kh):
    assert kh.khop_version() >= 10000
    for code in range(8):
        assert kh.strerror(code) and kh.strerror(code) != "unknown status"
    assert kh.strerror(99) == "unknown status"


def test_argument_checks_need_no_device(kh):
    L = kh.lib()
    out = ctypes.c_void_p()
    rp = (ctypes.c_uint32 * 4)(0, 1, 2, 3)
    ci = (ctypes.c_uint32 * 3)(1, 2, 0)
    assert L.khop_graph_create(3, rp, 4, ci, 3, 0, None, None) == kh.EINVAL      # no out
    assert L.khop_graph_create(0, rp, 4, ci, 3, 0, None, ctypes.byref(out)) == kh.EINVAL
    assert L.khop_graph_create(3, rp, 3, ci, 3, 0, None, ctypes.byref(out)) == kh.EINVAL
    assert L.khop_graph_create(3, None, 4, ci, 3, 0, None, ctypes.byref(out)) == kh.EINVAL
    assert L.khop_graph_create(3, rp, 4, ci, 3, 1 << 9, None, ctypes.byref(out)) == kh.EINVAL
    assert L.khop_graph_create(1 << 32, rp, 8, ci, 3, 0, None, ctypes.byref(out)) == kh.EINVAL
    assert L.khop_count(None, None, 1, 1, None, None) == kh.EINVAL
    assert L.khop_count_mixed(None, None, None, 1, None, 0, None) == kh.EINVAL
    assert L.khop_count_ex(None, None, None, 1, None, None, None, None, 0, None) == kh.EINVAL
    assert L.khop_get_error(None, None) == kh.EINVAL
    assert L.khop_graph_destroy(None) == kh.EINVAL
    assert L.khop_graph_set_tuning(None, None) == kh.EINVAL
    assert L.khop_submit(None, None, 0, 1, None) == kh.EINVAL
    assert L.khop_poll(None, None, 0, None, 0) == kh.EINVAL
    assert L.khop_server_destroy(None) == kh.EINVAL
    assert L.khop_server_create(None, None) == kh.EINVAL
    assert L.khop_batch_stats(None, None, None, None, None) == kh.EINVAL
    # the allocation-free entry point checks its limits first
    assert L.khop_count_static(0, rp, ci, None, None, 3, rp, 1, 1, rp, None) == kh.EINVAL
    assert L.khop_count_static((1 << 20) + 1, rp, ci, None, None, 3, rp, 1, 1, rp, None) == kh.EINVAL
    assert L.khop_count_static(3, rp, ci, None, None, (1 << 26) + 1, rp, 1, 1, rp, None) == kh.EINVAL
    assert L.khop_count_static(3, rp, ci, rp, None, 3, rp, 1, 1, rp, None) == kh.EINVAL


def test_graph_create_without_a_device_fails_loudly(kh):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    L = kh.lib()
    out = ctypes.c_void_p()
    rp = (ctypes.c_uint32 * 4)(0, 1, 2, 3)
    ci = (ctypes.c_uint32 * 3)(1, 2, 0)
    assert L.khop_graph_create(3, rp, 4, ci, 3, 0, None, ctypes.byref(out)) in (kh.ECUDA, kh.ENOMEM)
    assert not out.value
    srv = ctypes.c_void_p()
    assert L.khop_server_create(None, ctypes.byref(srv)) in (kh.ECUDA, kh.ENOMEM)


def test_binding_constants_match_the_header(kh):
    """Every KHOP_* enum value and flag of include/khop.h has the same value
    under the same name (without the prefix) in the binding."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    pairs = re.findall(r"\b(KHOP_(?:MODE|DIR)_\w+|KHOP_(?:REVERSE|UNDIRECTED|VALIDATE|SYMMETRIC))\s*=\s*(\d+)", src)
    assert pairs
    for name, value in pairs:
        py = name[len("KHOP_"):]
        assert hasattr(kh, py), py
        assert getattr(kh, py) == int(value), name
    modes = {n: int(v) for n, v in pairs if n.startswith("KHOP_MODE_")}
    assert modes["KHOP_MODE_BATCHED256"] == 4 and len(set(modes.values())) == len(modes)
