"""chan_rhs_terms_noalloc against the allocating chan_rhs_terms.

The scratch-free entry point serves callers that cannot allocate device
memory at the point of the call (a foreign memory pool, a latency-bound
loop, an arena that already owns the GPU): they pass device buffers for
H and N, and the only scratch is a fixed array inside the library.  This
file is collected last so that a failure here does not hide the others.
"""
import ctypes
import math

import numpy as np
import pytest

import synthetic as SY

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the parity tolerance of the other GPU tests (relative L2 per field)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_rhs_terms_noalloc_matches_allocating_entry_point(prec):
    """Every precision mode: H and N are FP64 complex fields in the caller's buffers
    whatever the handle stores.  In the pair-stored modes (2, 3) chan_rhs_terms runs its
    D1 sweep in FP32 pairs (~2^-47) and this entry point in FP64, which stays far inside
    the 1e-10 bar.  The second call must not change the device's free memory."""
    import torch
    import paper_1808_06461_b300 as chan
    lib = chan.library()
    args = (180.0, math.pi, math.pi / 2, 32, 49, 32, 1e-3)
    ch = chan.Channel(*args, precision=prec)
    y = ch.grid()
    n = ch.Ny * ch.Nz * ch.nxh
    out = torch.empty(2 * n * 2, dtype=torch.float64, device="cuda")
    for seed in (21, 22):   # two calls in a row, on different states
        s0 = SY.perturbed_poiseuille(y, 180.0, args[1], args[2], 32, 32, seed=seed, amp=0.1)
        ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        N_ref = ch.rhs_terms()
        H = ch.nonlinear()
        H_dev = torch.from_numpy(np.ascontiguousarray(H).view(np.float64).reshape(-1)).cuda()
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = lib.chan_rhs_terms_noalloc(ch.h, ctypes.c_void_p(H_dev.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert rc == chan.CHAN_OK, lib.chan_last_error(ch.h).decode()
        assert lib.chan_sync(ch.h) == chan.CHAN_OK
        if seed == 22:   # the first call of the process may load the library's module
            assert torch.cuda.mem_get_info()[0] == free0
        N = out.cpu().numpy().view(np.complex128).reshape((2,) + ch.shape)
        for f in range(2):
            assert _rel(N[f], N_ref[f]) < TOL, (prec, seed, f, _rel(N[f], N_ref[f]))
    ch.close()


def test_rhs_terms_noalloc_rejects_boxes_beyond_its_scratch():
    import torch
    import paper_1808_06461_b300 as chan
    lib = chan.library()
    ch = chan.Channel(180.0, math.pi, math.pi / 2, 256, 129, 256, 1e-3)   # 129 * 256 * 128 > 2097152
    buf = torch.empty(16, dtype=torch.float64, device="cuda")
    rc = lib.chan_rhs_terms_noalloc(ch.h, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()))
    assert rc == chan.CHAN_EINVAL
    assert "32 MiB" in lib.chan_last_error(ch.h).decode()
    ch.close()
