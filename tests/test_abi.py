"""The C ABI library loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bootmmpm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("bm_keygen", "bm_encrypt", "bm_bootstrap_batch", "bm_decrypt",
                 "bm_blind_rotate", "bm_sample_extract", "bm_key_switch"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2310_12441_gb300 import api
    lib = api.load()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(api.SYMBOLS) == set(_declared())


def test_status_strings():
    from paper_2310_12441_gb300 import api
    lib = api.load()
    assert lib.bm_status_str(0) == b"ok"
    assert lib.bm_status_str(-4) == b"look-up table is not negacyclic"


def test_null_arguments_are_rejected_on_host():
    from paper_2310_12441_gb300 import api
    lib = api.load()
    assert lib.bm_keygen(None, None, 0, None, None) == -1
    assert lib.bm_encrypt(None, 8, 2, None, None, None, 0, None) == -1
    assert lib.bm_workspace_bytes(None, 0, None, 0) == 0
    assert lib.bm_bootstrap_batch(None, 0, None, 0, None, None, None, None, 0, None) == -1


def test_job_struct_layout_matches_header():
    from paper_2310_12441_gb300 import api
    assert api.JOB_DTYPE.itemsize == 40
    assert api.JOB_DTYPE.fields["in_off"][1] == 16


def test_kernel_shape_table():
    """The autotuner's kernel shapes that fit each ring degree (host-side
    query), and refusal of shapes that do not fit."""
    from paper_2310_12441_gb300 import api
    api.load()
    assert set(api.kernel_shapes(1024)) == {0, 1, 2, 3, 4}
    assert set(api.kernel_shapes(2048)) == {0, 1, 2, 3, 4}
    assert set(api.kernel_shapes(4096)) == {0, 1, 2, 3, 4}
    assert set(api.kernel_shapes(8192)) == {0, 1}
    assert set(api.kernel_shapes(256)) == {0}
    assert api.kernel_shapes(16384) == {}
    assert api.kernel_shapes(1024)[1] == (8, 1024, 1)
    with pytest.raises(api.BMError):
        api.set_kernel_shape(8192, 2)
    with pytest.raises(api.BMError):
        api.set_kernel_shape(1000, 0)
    api.set_kernel_shape(2048, 4)
    assert api.get_kernel_shape(2048) == 4
    api.set_kernel_shape(2048, api.SHAPE_DEFAULT)
    assert api.get_kernel_shape(2048) == 1
    api.set_kernel_shape(256, api.SHAPE_DEFAULT)
    assert api.get_kernel_shape(256) == 0
