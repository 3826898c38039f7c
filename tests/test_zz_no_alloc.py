"""me_select_static: the selection with its tile counts in the library's
file-scope device array instead of caller scratch.  Two calls in a row (the
second reusing the array the first filled) must each equal me_select; sizes
above ME_SELECT_STATIC_MAX_PIX are refused before any device work."""
import ctypes

import numpy as np
import pytest

MAX_PIX = 1 << 24
ME_EINVAL = -1


def test_static_select_rejects_oversize():
    from paper_1208_0302_gb300 import _lib
    lib = _lib.load()
    cnt = ctypes.c_int(0)
    rc = lib.me_select_static(None, MAX_PIX + 1, 1, None, ctypes.cast(ctypes.byref(cnt), ctypes.c_void_p), None)
    assert rc == ME_EINVAL
    assert b"ME_SELECT_STATIC_MAX_PIX" in lib.me_last_error()
    rc = lib.me_select_static(None, -1, 1, None, ctypes.cast(ctypes.byref(cnt), ctypes.c_void_p), None)
    assert rc == ME_EINVAL


def test_header_limit_matches():
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "include", "genesis.h")).read()
    m = re.search(r"#define ME_SELECT_STATIC_MAX_PIX \(1 << (\d+)\)", src)
    assert m and (1 << int(m.group(1))) == MAX_PIX


@pytest.mark.gpu
def test_static_select_matches_select_twice_in_a_row(gpu):
    import torch
    rng = np.random.default_rng(2024)
    cases = [(rng.random(70001) < 0.4).astype(np.int32), (rng.random(2049) < 0.9).astype(np.int32),
             (rng.random(MAX_PIX) < 0.05).astype(np.int32)]
    for f in cases:
        ft = torch.tensor(f, device="cuda")
        ref_i, ref_c = gpu.select(ft, 1)
        for _ in range(2):  # two calls in a row share the static array
            idx, cnt = gpu.select_static(ft, 1)
            n = int(cnt.item())
            assert n == int(ref_c.item()) == int(f.sum())
            assert torch.equal(idx[:n], ref_i[:n])
