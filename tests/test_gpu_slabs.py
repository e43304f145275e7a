"""The plane-local transform passes run slab by slab through slab-sized buffers
(chan_opts.slab_planes), the implicit-step tables can be kept for one
substep only and recomputed each substep, or recomputed together with the
Poisson factors into work fields that are dead at that point of the substep
(chan_opts.lean_tables 1 and 2), and the
sweeps can read their mode-independent tables in place instead of staging
them in shared memory (chan_opts.y_tables).  Every kernel is plane-local in
those passes, the wall-normal kernels see the same full fields, and the
recomputed or relocated tables are the same numbers, so every combination
must give bitwise the same substeps, filter outputs, filtered pressure,
database record and statistics."""
import math

import numpy as np
import pytest

import oracle as O
import synthetic as SY

pytestmark = pytest.mark.gpu

CASES = {
    # Ny = 49 in 7 slabs of 7; Ny = 33 in slabs of 10, 10, 10 and a ragged 3
    "re180_32x49x32": ((180.0, math.pi, math.pi / 2, 32, 49, 32, 1e-3), 7),
    "re250_24x33x36": ((250.0, 2.0, 1.3, 24, 33, 36, 1e-3), 10),
}


def _run(chan, cfg, prec, slab, lean=-1, ytab=2):
    re, Lx, Lz, Nx, Ny, Nz, dt = cfg
    st = O.Setup(*cfg)
    s0 = SY.perturbed_poiseuille(st.y, re, Lx, Lz, Nx, Nz, seed=5, amp=0.1)
    ch = chan.Channel(*cfg, precision=prec, slab_planes=slab, lean_tables=lean, y_tables=ytab)
    ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    ch.step(4)
    ch.step(3)   # graph replay of a whole RK3 step from phase 1, then a partial one
    out = dict(ch.get_state())
    out["H"] = ch.nonlinear()
    out["ubar"], out["tau"] = ch.filter_stresses(1, 50.0, 50.0)
    out["stats"] = ch.stats()[0]
    out["ens"] = ch.filtered_enstrophy(0, 120.0, 60.0)
    out["p"] = ch.filtered_pressure(1, 50.0, 50.0)
    out["rec"] = ch.database_record(120.0, 60.0)
    ch.close()
    return out


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("name", list(CASES))
def test_slabs_and_lean_tables_are_bitwise_invisible(name, prec):
    import paper_1808_06461_b300 as chan
    cfg, slab = CASES[name]
    whole = _run(chan, cfg, prec, 0)
    for variant in ((slab, -1), (0, 1), (slab, 1), (0, -1, 1), (slab, 1, 1), (0, 2), (slab, 2, 1)):
        other = _run(chan, cfg, prec, *variant)
        for k in whole:
            assert np.array_equal(whole[k], other[k]), (name, prec, variant, k)
    assert np.isfinite(whole["v"]).all() and np.abs(whole["tau"]).max() > 0


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_tables_in_the_work_fields_take_no_memory_of_their_own(prec):
    """lean_tables = 2 drops the Poisson factors [Ny][7][C] and the one-substep Helmholtz tables
    [Ny][11][C] (C = Nz/2 * Nx/2 wavenumber classes) and adds the mean-flow solve's copies of
    their (0,0) class [3][Ny][11] and of H_1, H_3 at (0,0) [2][Ny]; in the pair-stored
    precisions it is lean_tables = 1."""
    import paper_1808_06461_b300 as chan
    cfg, _ = CASES["re180_32x49x32"]
    Nx, Ny, Nz = cfg[3], cfg[4], cfg[5]
    b = {}
    for lean in (1, 2):
        ch = chan.Channel(*cfg, precision=prec, lean_tables=lean, keep_rhs=-1)
        b[lean] = ch.device_bytes()
        ch.close()
    C = (Nz // 2) * (Nx // 2)
    saved = 18 * Ny * C * 8 - 33 * Ny * 8 - 2 * Ny * 16
    assert b[1] - b[2] == (0 if prec in (2, 3) else saved)
