"""The C-ABI library builds, loads without a GPU, exports every entry point
declared in include/*.h, and rejects bad arguments before touching CUDA."""
import ctypes
import glob
import os
import re

import pytest

from paper_2606_00817_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(ddf_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_2606_00817_gb300 import ddf
    return ddf.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ddf_create", "ddf_load_weights", "ddf_query_rays", "ddf_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2606_00817_gb300 import ddf
    raw = ctypes.CDLL(ddf.LIB_PATH)
    for name in _declared():
        assert hasattr(raw, name), name
        assert name in ddf.SIGNATURES, f"binding lacks {name}"


def test_param_count_and_bad_configs(lib):
    from paper_2606_00817_gb300 import ddf
    from paper_2606_00817_gb300.inputs import NetShape
    cfg = ddf.make_config(10, 1280, 8, "bf16")
    assert ddf.ddf_param_count(cfg) == NetShape(10, 1280, 8).n_params == 11_642_882
    assert ddf.ddf_param_count(ddf.make_config(6, 128, 4, "fp32")) == NetShape(6, 128, 4).n_params
    for bad in [ddf.make_config(-1, 128, 4), ddf.make_config(6, 100, 4), ddf.make_config(6, 128, 0),
                ddf.make_config(17, 128, 4), ddf.Config(6, 128, 4, 9, 0)]:
        assert ddf.ddf_param_count(bad) == 0
        with pytest.raises(ddf.DDFError) as e:
            ddf.ddf_create(bad)
        assert e.value.status == 1


def test_null_arguments_are_rejected(lib):
    from paper_2606_00817_gb300 import ddf
    assert lib.ddf_destroy(None) == 0
    assert lib.ddf_create(None, None) == 1
    arr = (ctypes.c_void_p * 6)()
    rp = ctypes.cast(arr, ddf._RAYS)
    assert lib.ddf_query_rays(None, rp, 10, None, None, None) == 1
    assert "NULL" in ddf.ddf_last_error()
    assert lib.ddf_set_chunk_rays(None, 1024) == 1
    assert lib.ddf_check_status(None, None) == 1
