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


def test_init_rejects_a_negative_slab():
    lib = chan.library()
    o = chan.chan_opts()
    lib.chan_opts_default(ctypes.byref(o))
    o.re_tau, o.Lx, o.Lz, o.Nx, o.Ny, o.Nz, o.dt = 180.0, 3.14, 1.57, 32, 49, 32, 1e-3
    o.slab_planes = -1
    h = ctypes.c_void_p()
    assert lib.chan_init_ex(ctypes.byref(h), ctypes.byref(o)) == chan.CHAN_EINVAL
    assert not h.value
    assert "slab" in lib.chan_last_error(None).decode()


def test_footprint_of_the_large_grids():
    """The transform buffers are slab-sized: the Re_tau 1000 grid (768 x 385 x 768) in FP64 and
    in mixed precision stays below 65 GB; the 12 mixed fields of one slab stay below 8 GiB."""
    for prec in (chan.CHAN_PREC_FP64, chan.CHAN_PREC_MIXED):
        assert chan.footprint_bytes(768, 385, 768, prec) < 65e9
    # the Re_tau 2000 box (1536 x 633 x 1152, mixed) with the per-substep tables computed into
    # dead work fields and no kept Helmholtz right-hand sides, both chosen automatically, and
    # the filter pass in slabs within 4 GiB
    assert chan.footprint_bytes(1536, 633, 1152, chan.CHAN_PREC_MIXED) < 150e9
    # the slab share of the footprint: FP64 384 x 257 x 384 holds all 257 planes at once
    small = chan.footprint_bytes(384, 257, 384, chan.CHAN_PREC_FP64)
    n = 257 * 384 * 192
    assert small > (6 + 18) * n * 16 + 12 * 257 * 576 * 192 * 16


def test_init_rejects_an_unknown_precision():
    lib = chan.library()
    o = chan.chan_opts()
    lib.chan_opts_default(ctypes.byref(o))
    o.re_tau, o.Lx, o.Lz, o.Nx, o.Ny, o.Nz, o.dt = 180.0, 3.14, 1.57, 32, 49, 32, 1e-3
    o.precision = 4
    h = ctypes.c_void_p()
    assert lib.chan_init_ex(ctypes.byref(h), ctypes.byref(o)) == chan.CHAN_EINVAL
    assert not h.value
    assert "precision" in lib.chan_last_error(None).decode()


def test_footprint_orders_the_modes():
    """Pair storage adds the pair copies of the implicit-step tables; FP32 transforms halve
    the mixed-layout fields.  Same box, same slab choice: FP64 < F64X and MIXED < MIXED_DF."""
    for args in ((384, 257, 384), (96, 97, 64)):
        f = [chan.footprint_bytes(*args, p) for p in range(4)]
        assert f[chan.CHAN_PREC_FP64] < f[chan.CHAN_PREC_F64X]
        assert f[chan.CHAN_PREC_MIXED] < f[chan.CHAN_PREC_MIXED_DF]


def test_init_rejects_an_unknown_table_placement():
    lib = chan.library()
    o = chan.chan_opts()
    lib.chan_opts_default(ctypes.byref(o))
    o.re_tau, o.Lx, o.Lz, o.Nx, o.Ny, o.Nz, o.dt = 180.0, 3.14, 1.57, 32, 49, 32, 1e-3
    o.y_tables = 3
    h = ctypes.c_void_p()
    assert lib.chan_init_ex(ctypes.byref(h), ctypes.byref(o)) == chan.CHAN_EINVAL
    assert "y_tables" in lib.chan_last_error(None).decode()


def test_every_traced_kernel_id_has_a_name():
    """The binding's CHAN_NKERNELS is the header's and the library's: chan_kernel_name names
    ids 0 .. CHAN_NKERNELS - 1 (distinct names) and no id past them."""
    lib = chan.library()
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "chan.h")).read()
    assert int(re.search(r"#define CHAN_NKERNELS (\d+)", hdr).group(1)) == chan.CHAN_NKERNELS
    names = [lib.chan_kernel_name(k) for k in range(chan.CHAN_NKERNELS)]
    assert all(n is not None for n in names)
    assert len(set(names)) == chan.CHAN_NKERNELS
    assert lib.chan_kernel_name(chan.CHAN_NKERNELS) is None
    assert lib.chan_kernel_name(-1) is None
    assert b"k_setup_pois" in names and b"k_copy_mean_modes" in names
