"""The C-ABI library loads and exports every entry point that include/*.h declares (no GPU).

No compute call is made here; calls that fail argument checks before touching the GPU are fine.
"""
import ctypes
import glob
import os
import re

import pytest

from paper_1812_07122_gb300 import blfls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_07122_gb300 import build
    build.build()
    return blfls.load()


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(blfls_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["blfls_create", "blfls_smooth", "blfls_destroy", "blfls_last_error",
                     "blfls_smooth_host", "blfls_blf_residual", "blfls_solve_residual",
                     "blfls_smooth_batch"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_covers_every_declared_symbol():
    assert _declared_functions() <= set(blfls.exported_symbols())


def test_null_handle_is_rejected_without_touching_the_gpu(lib):
    rc = lib.blfls_smooth(None, 1, 1, 8, 8, 1, 1.0, 1.0, 0.1, 1, 1, 0, None)
    assert rc == blfls.BLFLS_EINVAL
    assert "handle" in blfls.blfls_last_error()
    with pytest.raises(blfls.BlflsError) as ei:
        blfls.blfls_smooth(None, 1, 1, 8, 8, 1, 1.0, 1.0, 0.1, 1)
    assert ei.value.code == blfls.BLFLS_EINVAL


def test_create_rejects_null_out(lib):
    assert lib.blfls_create(None, 0, 0, None) == blfls.BLFLS_EINVAL


def test_destroy_is_null_safe(lib):
    lib.blfls_destroy(None)


def test_job_struct_matches_the_header():
    # pointer, pointer, 3 ints, 3 floats, 3 ints
    ps = ctypes.sizeof(ctypes.c_void_p)
    assert ctypes.sizeof(blfls.blfls_job) == 2 * ps + 9 * 4 + (4 if ps == 8 else 0)


@pytest.mark.parametrize("name,args", [
    ("blfls_smooth_host", (1, 1, 8, 8, 1, 1.0, 1.0, 0.1, 1, 1, 0, None)),
    ("blfls_smooth_ls", (1, 1, 8, 8, 1, 1.0, 1, None)),
    ("blfls_layers", (1, 1, 8, 8, 1, 0, 2.0, 1.0, 1.0, 0.1, 1, 1, 0, None)),
    ("blfls_gaussian", (1, 1, 8, 8, 1, 1.0, None)),
    ("blfls_smooth_guided", (1, 1, 1, 8, 8, 1, 1, 1.0, 1.0, 0.1, 1, 1, 0, None)),
    ("blfls_smooth_rolling", (1, 1, 8, 8, 1, 1.0, 1.0, 0.1, 1, 1, 1.0, 0, None)),
    ("blfls_smooth_grid", (1, 1, 8, 8, 1, 1.0, 1.0, 0.1, 1, None)),
    ("blfls_smooth_nc", (1, 1, 8, 8, 1, 1.0, 1.0, 0.1, 1, 3, None)),
    ("blfls_smooth_normalized", (1, 1, 8, 8, 1, 1.0, 1.0, 0.1, 1, 1, 0, None)),
    ("blfls_blf_residual", (1, 1, 1, 8, 8, 1, 1.0, 0.1, 1, 0, None)),
    ("blfls_solve_residual", (1, 1, 1, 1, 8, 8, 1, 1.0, None)),
    ("blfls_smooth_batch", (None, 0, None)),
    ("blfls_profile_begin", (16,)),
    ("blfls_submit", (None, None)),
    ("blfls_poll", (1, None)),
])
def test_every_entry_point_rejects_a_null_handle_on_the_host(lib, name, args):
    """Argument checks run on the host before anything touches the GPU: a NULL handle is
    BLFLS_EINVAL from every entry point that takes one."""
    assert getattr(lib, name)(None, *args) == blfls.BLFLS_EINVAL


def test_device_checks_reject_a_null_word_on_the_host(lib):
    assert lib.blfls_device_checks(0, None) == blfls.BLFLS_EINVAL
