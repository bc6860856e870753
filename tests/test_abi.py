"""The C-ABI library loads, exports every function include/dpv.h declares,
and reports errors through status codes and dpvGetLastError (no GPU needed:
no call here launches work)."""
import ctypes as C
import os
import re

import pytest

from paper_2407_00179_b300 import build, dpv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dpv.h")).read()
    return sorted(set(re.findall(r"^\s*(?:dpv_status|const char\*)\s+(dpv\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return dpv.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(dpv.EXPORTS)


# The calls of the boundary the scope table fixes (device creation, per-rank
# commit, globally consistent TF / cameras / frame, collaborative render,
# frame ready, frame and fragment maps, order map, backward, last error,
# release): every one is declared and exported.
SCOPE_CALLS = ["dpvCreateDevice", "dpvSetVolumeGeometry", "dpvCommitBrick", "dpvSetTransferFunction",
               "dpvSetCameras", "dpvSetFrame", "dpvRenderFrame", "dpvFrameReady", "dpvMapFrame", "dpvUnmapFrame",
               "dpvMapFragments", "dpvMapOrder", "dpvBackward", "dpvGetLastError", "dpvRelease"]


def test_exports_every_scope_call(lib):
    names = _declared()
    for n in SCOPE_CALLS:
        assert n in names, n
        assert hasattr(lib, n), n


def test_every_declaration_cites_or_disclaims_a_passage():
    """Each declaration's comment names the passage of the paper it follows
    (a section sign) or says the paper has no counterpart."""
    src = open(os.path.join(ROOT, "include", "dpv.h")).read()
    body = src[src.index("typedef struct dpv_device_t"):]
    missing = []
    for m in re.finditer(r"^\s*(?:dpv_status|const char\*)\s+(dpv\w+)\s*\(", body, re.M):
        # the comment block(s) right above the declaration (a pair such as
        # map / unmap may share one)
        before = body[:m.start()]
        cstart = before.rfind("/*")
        comment = re.sub(r"\s*\n\s*\*?\s*", " ", before[cstart:])
        if "§" not in comment and "no counterpart" not in comment and "not in the paper" not in comment:
            missing.append(m.group(1))
    assert not missing, missing


def test_null_and_bad_arguments(lib):
    assert lib.dpvRelease(None) == 0
    h = C.c_void_p()
    assert lib.dpvCreateDevice(0, 0, None, C.byref(h)) == 1          # DPV_ERR_INVALID_ARG
    assert b"num_ranks" in lib.dpvGetLastError()
    assert lib.dpvCreateDevice(256, 0, None, C.byref(h)) == 1
    assert lib.dpvCreateDevice(1, 0, None, None) == 1
    assert lib.dpvRenderFrame(None) == 1
    assert lib.dpvSetFrame(None, None) == 1


def test_struct_layouts_match_header():
    # dpv_brick_desc: 6 ints, dtype, float, dtype, pointer, 6 ints, int
    assert C.sizeof(dpv.BrickDesc) == 4 * 9 + 4 + 8 + 4 * 7 + 4
    assert C.sizeof(dpv.CameraDesc) == 40
    assert C.sizeof(dpv.FrameDesc) == 36
    assert C.sizeof(dpv.Stats) == 40 + 8 * 6 + 4 * 6 + 8 + 8 + 8


def test_no_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = lib.dpvCreateDevice(1, 0, None, C.byref(h))
    assert st == 4 and not h.value                                   # DPV_ERR_CUDA
