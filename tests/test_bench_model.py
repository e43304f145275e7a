"""The bench's algorithmic flop model (the numerator of its roofline fraction), checked
against an explicit walk over the butterflies of both stage orderings the library uses:
decimation in frequency (twiddle of butterfly j in a block of span m is 1 when j = 0) and
the Cooley-Tukey inverse with natural input (twiddle of block b is 1 when the digit reversal
of b is 0).  A radix-R butterfly costs its DFT additions plus (R - 1) complex products of 6
flops unless its twiddle is 1; the pruned first stage of a padded inverse and the pruned last
stage of a truncated forward transform cost 12 and 14 (13 each on average)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_model", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


DFT = {2: 4, 3: 16, 4: 16}


def walk_dif(plan, L):
    tot, Ls = 0.0, L
    for s, R in enumerate(plan):
        m = Ls // R
        for blk in range(L // Ls):
            for j in range(m):
                d = 13.0 if s == 0 else DFT[R]
                tot += d + (6 * (R - 1) if j > 0 else 0)
        Ls //= R
    return tot


def digit_reversal(b, plan, s):
    K, w = 0, 1
    for i in range(s):
        w *= plan[i]
    for i in range(s - 1, -1, -1):
        w //= plan[i]
        K += (b % plan[i]) * w
        b //= plan[i]
    return K


def walk_ct_inverse(plan, L):
    tot, Ls = 0.0, L
    for s, R in enumerate(plan):
        m = Ls // R
        for blk in range(L // Ls):
            K = digit_reversal(blk, plan, s)
            for j in range(m):
                d = 13.0 if s == 0 else DFT[R]
                tot += d + (6 * (R - 1) if K > 0 else 0)
        Ls //= R
    return tot


@pytest.mark.parametrize("L", [6, 12, 18, 36, 48, 72, 96, 576, 864, 1152, 1728, 2304])
def test_fft_flop_model_matches_both_orderings(bench, L):
    plan = bench.radix_plan(L)
    model = bench.fft_flops(L)
    assert walk_dif(plan, L) == model
    assert walk_ct_inverse(plan, L) == model


def test_digit_reversal_is_a_permutation():
    plan = [3, 3, 4, 4, 4]
    for s in range(1, len(plan) + 1):
        n = 1
        for r in plan[:s]:
            n *= r
        assert sorted(digit_reversal(b, plan, s) for b in range(n)) == list(range(n))


def test_xpass_flops_of_the_bench_workload(bench):
    c = dict(Nx=384, Ny=257, Nz=384)
    L1, L3, nxh = 576, 576, 192
    pairs = c["Ny"] * L3 // 2
    assert bench.kernel_flops("k_xpass", c, {}) == pairs * (9 * bench.fft_flops(L1) + L1 * 18 + 3 * nxh * 16)


def test_step_bytes_match_the_per_point_budget(bench):
    """The byte model per collocation point and substep (pt = Nx Ny Nz, a mode-point is two
    pts): in FP64 the transform passes move a1 56, a2 120 (six inputs; a budget that counts
    omega_2's load under a1 gives 112), a3 108 and a4 60 bytes per pt, and the FP32 transforms
    of the mixed modes halve the physical-layout fields."""
    c = dict(Nx=384, Ny=257, Nz=384)
    pts = 384 * 257 * 384
    b = bench.step_bytes(c, "fp64", 1, filtered=False)
    per = {k: v / pts for k, v in b.items()}
    assert per["k_pre"] == 56 and per["k_zinv"] == 120 and per["k_xpass"] == 108 and per["k_zfwd"] == 60
    assert per["k_nonlin"] == 40
    m = bench.step_bytes(c, "mixed", 1, filtered=False)
    assert m["k_xpass"] / pts == 54 and m["k_zinv"] / pts == 16 + 16 + 36
    # the filter pass adds work only when asked, and more of it than one substep's transforms
    f = bench.step_bytes(c, "fp64", 1)
    assert f["k_zfwd"] > b["k_zfwd"] and "k_filter_out" in f and "k_filter_out" not in b
