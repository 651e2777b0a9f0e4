"""The C-ABI library builds, loads and exports every entry point that
include/lcc.h declares (no GPU needed; no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lcc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lcc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_06972_gb300 import build, lcc
    build.build()
    return lcc.load()


def test_header_declares_the_paper_calls():
    names = _declared()
    for n in ("lcc_encode_keyframe", "lcc_encode_pframe", "lcc_decode", "lcc_create", "lcc_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2008_06972_gb300 import lcc
    for n in _declared():
        assert hasattr(lib, n), n
    assert sorted(lcc.exported_symbols()) == sorted(_declared())


def test_status_strings_and_defaults(lib):
    from paper_2008_06972_gb300 import lcc
    assert lcc.status_string(lcc.OK) == "ok"
    assert lcc.status_string(lcc.ERR_CORRUPT) == "corrupt stream"
    p = lcc.default_params()
    assert (p.tile_h, p.tile_w, p.max_refits, p.merge_runs) == (4, 4, 3, 1)
    assert abs(p.fit_thr_m - 0.05) < 1e-9 and abs(p.quant_m - 0.02) < 1e-9


def test_create_without_gpu_reports_no_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2008_06972_gb300 import lcc
    import synth
    with pytest.raises(lcc.LccError) as e:
        lcc.Context(synth.CFG1_SENSOR)
    assert e.value.status in (lcc.ERR_NO_DEVICE, lcc.ERR_CUDA)


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA sources include nothing from each other."""
    csrc = os.path.join(ROOT, "paper_2008_06972_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower() or f.endswith(".md"), f
    orc = open(os.path.join(ROOT, "oracle", "lcc_oracle.c")).read()
    assert "lcc_internal" not in orc and "lcc.h" not in orc.replace("lcc_oracle.h", "")
