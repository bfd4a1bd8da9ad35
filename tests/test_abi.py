"""The C-ABI library builds, loads without a GPU, and exports every function that
include/sst.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sst.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:sst_status|const char\*)\s+(sst_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import shutil
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_2101_11489_gb300 import _build
    return ctypes.CDLL(_build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("sst_create", "sst_destroy", "sst_calib_upload", "sst_unpack", "sst_cluster", "sst_batch",
                 "sst_autotune", "sst_submit", "sst_poll", "sst_server_start", "sst_server_stop", "sst_last_error"):
        assert want in names


def test_library_exports_every_declared_function(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_function(lib):
    import paper_2101_11489_gb300 as sst
    assert set(declared_functions()) == set(sst.exported_symbols())
    sst.load_library()


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    import paper_2101_11489_gb300 as sst
    L = sst.load_library()
    assert L.sst_create(None, 0, 1) == sst.SST_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert L.sst_create(ctypes.byref(h), 0, 0) == sst.SST_ERR_INVALID_ARG
    assert L.sst_destroy(None) == sst.SST_ERR_INVALID_ARG
    assert L.sst_last_error(None) == b"null context"


def test_status_bits_agree_between_header_binding_and_oracle():
    """The data-error bits are an interface: the header, the binding and the
    independently written oracle must report the same values."""
    import re
    import oracle as orc
    import paper_2101_11489_gb300 as sst
    hdr = open(os.path.join(ROOT, "include", "sst.h")).read()
    for name in ("FED_HDR", "FRAMING", "BAD_CODE", "RUN_RANGE", "RUN_ORDER", "TRUNC"):
        m = re.search(r"#define SST_CH_%s (0x[0-9A-Fa-f]+)u" % name, hdr)
        assert m, name
        assert int(m.group(1), 16) == getattr(sst, "SST_CH_" + name) == getattr(orc, "ST_" + name)


def test_binding_constants_agree_with_the_header():
    """Limits the binding checks on the host side are the header's."""
    import re
    import paper_2101_11489_gb300 as sst
    hdr = open(os.path.join(ROOT, "include", "sst.h")).read()
    m = re.search(r"#define SST_NOALLOC_MAX_FEDS (\d+)u", hdr)
    assert m and int(m.group(1)) == sst.NOALLOC_MAX_FEDS
    for name in ("OK", "ERR_INVALID_ARG", "ERR_NO_CALIB", "ERR_BUDGET", "ERR_TOO_LARGE", "ERR_BUSY",
                 "ERR_NOT_READY", "ERR_TIMEOUT", "ERR_CUDA", "ERR_STATE"):
        m = re.search(r"#define SST_%s (\d+)" % name, hdr)
        assert m and int(m.group(1)) == getattr(sst, "SST_" + name), name


def test_record_layouts_match_the_header():
    """The ctypes records mirror the header's structs field for field (all fields
    are 32- or 64-bit, so the sizes follow from the field lists)."""
    import paper_2101_11489_gb300 as sst
    assert ctypes.sizeof(sst.sst_tune) == 6 * 4
    assert ctypes.sizeof(sst.sst_launch_info) == 5 * 4
    assert ctypes.sizeof(sst.sst_event_status) == 16
