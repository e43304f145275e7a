"""The C-ABI library loads, exports every declared entry point, and rejects
bad arguments with CHAN_EINVAL before any device work (runs without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_1808_06461_b300 as chan

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "chan.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chan_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert len(names) >= 15
    lib = ctypes.CDLL(chan.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(chan.SYMBOLS) == names


@pytest.mark.parametrize("args,frag", [
    ((180.0, 3.14, 1.57, 30, 49, 32, 1e-3), "Nx"),          # 30 is not 2^a 3^b
    ((180.0, 3.14, 1.57, 32, 48, 32, 1e-3), "Ny"),          # even Ny
    ((180.0, 3.14, 1.57, 32, 49, 34, 1e-3), "Nz"),
    ((180.0, 3.14, 1.57, 32, 49, 32, 0.0), "dt"),
    ((-1.0, 3.14, 1.57, 32, 49, 32, 1e-3), "positive"),
    ((180.0, 3.14, 1.57, 1536, 49, 32, 1e-3), "too long"),   # FP64 x-pass does not fit shared memory
])
def test_init_rejects_bad_arguments(args, frag):
    lib = chan.library()
    h = ctypes.c_void_p()
    rc = lib.chan_init(ctypes.byref(h), *args)
    assert rc == chan.CHAN_EINVAL
    assert not h.value
    msg = lib.chan_last_error(None).decode()
    assert frag in msg


def test_null_handle_calls_fail_cleanly():
    lib = chan.library()
    assert lib.chan_step(None, 1) == chan.CHAN_EINVAL
    assert lib.chan_sync(None) == chan.CHAN_EINVAL
    assert lib.chan_fourier_count(None) == 0
    lib.chan_free(None)
