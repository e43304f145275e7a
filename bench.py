#!/usr/bin/env python
"""Throughput of the channel substep on B300: DNS Mpts.substep/s.

Workload (default): Re_tau = 550, Lx = 2 pi, Lz = pi, 384 x 257 x 384
collocation points, dt = 2e-4, FP64, seeded turbulent-like initial field
(Reichardt mean + k^-5/3 random-phase fluctuations).  One bench "step" is
one pass of the whole hot path: 50 RK3 substeps, then the filter with the
filtered stresses (sharp cut-off l1c+ = 120, l3c+ = 60), then the plane
statistics -- the cadence of that workload (filtered fields every 50
substeps).  Throughput counts N1 N2 N3 points x 50 substeps per step.

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 under
torch.distributed.run each rank runs an independent replica (the path has
no data exchange: weak scaling, replicas only).  ``--impl reference`` times
the FP64 CPU oracle on a bounded sample of the same workload instead.
"""
import argparse
import copy
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The serving leg keeps 16 runs on 16 streams; with the default 8 hardware work queues the
# streams alias and serialise (measured: the per-run-stream serving mix gains 9-34 %).  Read
# at context creation, so set before torch or the library touches the GPU.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np  # noqa: E402

CONFIGS = {
    "re550_384x257x384": dict(re=550.0, Lx=2 * math.pi, Lz=math.pi, Nx=384, Ny=257, Nz=384, dt=2e-4,
                              sub_per_step=50, filt=(0, 120.0, 60.0)),
    "re180_32x49x32": dict(re=180.0, Lx=math.pi, Lz=math.pi / 2, Nx=32, Ny=49, Nz=32, dt=1e-3,
                           sub_per_step=10, filt=(1, 50.0, 50.0)),
    # profiling case: the same x-z planes as the Re 550 workload with 33 wall-normal points
    # (inputs of one pass 0.35 GB > L2, about 2 GB on the device)
    "re550_384x33x384": dict(re=550.0, Lx=2 * math.pi, Lz=math.pi, Nx=384, Ny=33, Nz=384, dt=2e-4,
                             sub_per_step=10, filt=(0, 120.0, 60.0)),
    "re1000_768x385x768": dict(re=1000.0, Lx=2 * math.pi, Lz=math.pi, Nx=768, Ny=385, Nz=768, dt=1e-4,
                               sub_per_step=50, filt=(0, 120.0, 60.0)),
    # relaxed-resolution Re 2000 box, mixed precision only (3Nx/2 = 2304 exceeds the FP64
    # in-CTA transform); box filter of width 100 wall units every 20 substeps; about 147 GB
    # on the device (slabbed transforms, per-substep implicit tables in the work fields)
    "re2000_1536x633x1152": dict(re=2000.0, Lx=2 * math.pi, Lz=math.pi, Nx=1536, Ny=633, Nz=1152, dt=5e-5,
                                 sub_per_step=20, filt=(1, 100.0, 100.0)),
}
DEFAULT = "re550_384x257x384"


# ---------------------------------------------------------------------------
# Algorithmic FP64 flop counts of each kernel (per launch), from the steps the
# kernels take: in-place mixed-radix 3/4/2 FFTs (a radix-R butterfly costs its
# DFT adds plus (R-1) twiddle complex multiplies of 6 flops unless its twiddle
# index is 0) and the banded sweeps of the wall-normal solves (a real
# coefficient times a complex value = 2 FMA = 4 flops).
# ---------------------------------------------------------------------------
def radix_plan(L):
    """Decimation-in-frequency radix order of the library: 3s, then 4s, then one 2."""
    r, out = L, []
    while r % 3 == 0:
        out.append(3); r //= 3
    while r % 4 == 0:
        out.append(4); r //= 4
    while r % 2 == 0:
        out.append(2); r //= 2
    assert r == 1
    return out


def fft_flops(L, pruned=True):
    """Flops of one in-place mixed-radix transform of length L.

    Stage with block Ls and span m = Ls/R: L/R butterflies; each costs its DFT
    (radix 2: 4, radix 4: 16, radix 3: 16 flops) plus (R-1) twiddle complex
    multiplies (6 flops) unless j = 0 (a 1/m fraction).  (The inverse transforms
    run Cooley-Tukey stages whose twiddle-free butterflies are the first block of
    each stage instead; the count of twiddled butterflies is the same.)  With the 3/2 padding
    the first radix-3 stage of an inverse has a zero middle input (12 flops) and
    the last one of a forward transform skips its middle output (14 flops):
    both cost 13.5 on average over the pair, counted per transform as 12 + 14 / 2.
    """
    dft = {2: 4, 4: 16, 3: 16}
    tot, Ls = 0.0, L
    for s, R in enumerate(radix_plan(L)):
        m = Ls // R
        d = dft[R]
        if pruned and s == 0:
            d = 13.0
        tot += (L // R) * (d + (1.0 - 1.0 / m) * (R - 1) * 6)
        Ls //= R
    return tot


# DRAM bytes per wall-normal plane of each kernel launch, from ncu on the 384 x 33 x 384
# profiling case (profiles/k_xpass_fp64_re550_384x33x384.md: dram__bytes_read.sum +
# dram__bytes_write.sum divided by 33); valid for Nx = Nz = 384 only and only while the
# kernels are as captured (NCU_CURRENT).
NCU_BYTES_PER_PLANE = {("k_xpass", "fp64"): (350.522368e6 + 131.073536e6) / 33}
NCU_PIPE = {("k_xpass", "fp64"): ("fp64", 0.8963)}
NCU_CURRENT = {("k_xpass", "fp64"): True}


# per mode-point flops of the wall-normal kernels (read off their sweeps)
# (k_helm: the right-hand side from the previous substep's solve, A and no B product)
Y_FLOPS = {"k_pre": 140, "k_nonlin": 70, "k_helm": 136, "k_poisson": 132, "k_derive": 140}


def kernel_flops(name, c, launches_by_mode):
    Nx, Ny, Nz = c["Nx"], c["Ny"], c["Nz"]
    nxh, L1, L3 = Nx // 2, 3 * Nx // 2, 3 * Nz // 2
    M = nxh * Nz
    if name in Y_FLOPS:
        return Y_FLOPS[name] * M * Ny
    if name in ("k_zinv", "k_zfwd"):
        nf = launches_by_mode.get(name, 6 if name == "k_zinv" else 3)
        return nf * Ny * nxh * fft_flops(L3)
    if name == "k_xpass":
        pairs = Ny * L3 // 2
        return pairs * (9 * fft_flops(L1) + L1 * 18 + 3 * nxh * 16)
    return 0


def step_flops(c, nsub, filtered=True):
    """Algorithmic flops per bench step by kernel (nsub substeps, then the filter pass when
    ``filtered``): the per-launch counts of ``kernel_flops`` for the substep launches over all
    Ny planes, whatever slabs the transform passes run in, plus the filter pass's transforms
    (six inverse z columns, two x-passes of three inverse and six forward rows with the six
    products, twelve forward z columns) and its one k_pre."""
    Nx, Ny, Nz = c["Nx"], c["Ny"], c["Nz"]
    nxh, L1, L3 = Nx // 2, 3 * Nx // 2, 3 * Nz // 2
    out = {k: nsub * kernel_flops(k, c, {}) for k in ("k_pre", "k_zinv", "k_xpass", "k_zfwd", "k_nonlin",
                                                       "k_helm", "k_poisson")}
    if filtered:
        pairs = Ny * L3 // 2
        out["k_pre"] += kernel_flops("k_pre", c, {})
        out["k_zinv"] += 6 * Ny * nxh * fft_flops(L3)
        out["k_xpass"] += 2 * pairs * (9 * fft_flops(L1) + L1 * 12 + 6 * nxh * 16)
        out["k_zfwd"] += 12 * Ny * nxh * fft_flops(L3)
    return out


# ---------------------------------------------------------------------------
# Algorithmic HBM bytes: every field a kernel reads, once, and every field it
# writes, once, at the size the precision mode stores it; the wall-normal
# kernels also read their per-wavenumber-class tables once per class.  Scratch
# round trips (the forward sweeps parked for the backward sweeps) and re-reads
# are not counted: they are what measured DRAM traffic above this model shows.
# Per mode-point (n = Ny Nz Nx/2 of them per field):
#   F   = 16 B  a Fourier field (complex FP64, or an FP32 (hi, lo) pair per part)
#   fin = 8 B   the FP32 transform inputs u_1, u_3, omega_1, omega_3 (mixed modes), else 16
#   X   = 1.5 es  a field in the z-physical layout (3Nz/2 rows; es 8 B FP32, else 16)
#   tab = 8 B   a table value (FP64, or an FP32 pair)
# ---------------------------------------------------------------------------
def step_bytes(c, mode, nsub, filtered=True):
    """Algorithmic bytes per bench step (nsub substeps, then the filter pass and the
    statistics when ``filtered``), by kernel name."""
    Nx, Ny, Nz = c["Nx"], c["Ny"], c["Nz"]
    nxh = Nx // 2
    M = Nz * nxh
    C = (Nz // 2) * nxh
    n = Ny * M
    f32 = mode in ("mixed", "mixed_df")
    F, tab = 16.0, 8.0
    fin = 8.0 if f32 else 16.0
    X = 1.5 * (8.0 if f32 else 16.0)
    sub = {"k_pre": n * (3 * F + 4 * fin),
           "k_zinv": n * (4 * fin + 2 * F + 6 * X),
           "k_xpass": n * 9 * X,
           "k_zfwd": n * (3 * X + 3 * F),
           "k_nonlin": n * 5 * F,
           "k_helm": n * 14 * F + 7 * tab * Ny * C,
           "k_poisson": n * 4 * F + 11 * tab * Ny * C,
           "k_mean": 10 * 8.0 * Ny}
    out = {k: v * nsub for k, v in sub.items()}
    if filtered:
        fil = {"k_pre": n * 7 * F,
               "k_zinv": n * (6 * F + 6 * X) + 8.0 * M,
               "k_xpass": 2 * n * 9 * X,
               "k_zfwd": n * (12 * X + 12 * F),
               "k_filter_out": n * (15 * F + 9 * F),
               "k_stats": n * 12 * F}
        for k, v in fil.items():
            out[k] = out.get(k, 0.0) + v
    return out


# ---------------------------------------------------------------------------
def clocks_sampler(stop, out):
    cmd = ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-i", str(int(os.environ.get("LOCAL_RANK", "0")))]
    while not stop.is_set():
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=5)
            if r.returncode == 0 and r.stdout.strip():
                out.append([x.strip() for x in r.stdout.strip().splitlines()[0].split(",")])
        except Exception:
            pass
        stop.wait(0.2)


def summarize_clocks(samples):
    if not samples:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    sm = [float(s[0]) for s in samples if s[0].replace(".", "").isdigit()]
    mx = [float(s[1]) for s in samples if s[1].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for s in samples for i in range(4) if len(s) > 3 + i and s[3 + i] == "Active"})
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(samples)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except Exception:
        return {}


# FP64 ALU peak from unit counts and clocks: 148 SMs x 2 FP64 FMA lanes per SM per clock
# (the per-SM FP64 rate ncu reports for this part) x 2 flops x 2032 MHz maximum SM clock.
SMS, FP64_FMA_PER_SM_CLK, SM_MAX_MHZ = 148, 2, 2032.0
FP64_PEAK_DERIVED_TFLOPS = SMS * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
# FP32 ALU peak the same way: 128 FP32 FMA lanes per SM per clock (four 32-lane partitions).
FP32_FMA_PER_SM_CLK = 128
FP32_PEAK_DERIVED_TFLOPS = SMS * FP32_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12


def fp64_peak_tflops(torch):
    """Dense FP64 rate of this GPU, measured as a cuBLAS DGEMM (best of 3), TFLOP/s."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 1e9
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


# ---------------------------------------------------------------------------
# Replicas (N > 1 under torch.distributed.run): every rank runs its own box;
# the job's time is the slowest rank's and its throughput counts every rank.
# ---------------------------------------------------------------------------
def max_over_ranks(x, dist=None, device="cpu"):
    """Largest value of x over the ranks of the default process group (x itself alone)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, steps, substeps_per_step, points, max_ms):
    """Weak scaling: all ranks' point-substeps over the slowest rank's time, in Mpts.substep/s."""
    return world * steps * substeps_per_step * points / (max_ms * 1e-3) / 1e6


def workload_config(name, c, mode, world=1):
    """The ``config`` of a bench line: the same dict for our arm and the reference arm."""
    kind, p1, p3 = c["filt"]
    n = c["Ny"] * c["Nz"] * (c["Nx"] // 2)
    return {"workload": name, "Nx": c["Nx"], "Ny": c["Ny"], "Nz": c["Nz"], "re_tau": c["re"],
            "dt": c["dt"], "substeps_per_step": c["sub_per_step"],
            "filter": {"kind": "sharp" if kind == 0 else "box", "p1": p1, "p3": p3},
            "precision": mode,
            "l2": ("inputs larger than L2 (state %.1f GB)" % (6 * n * 16 / 1e9) if 6 * n * 16 > 126e6 else
                   "inputs within L2 (state %.1f MB): a small parity case, not a bandwidth measurement"
                   % (6 * n * 16 / 1e6)),
            "parallelism": "replicas" if world > 1 else "single"}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample_substep_seconds(c, n_planes=4, n_modes=512, with_filter=False):
    """Estimated oracle seconds per substep (and per filter pass) of the full workload, from a sample.

    Timed: the wall-normal derivatives of the a1 step over all modes, the
    a2-a4 transforms and products on ``n_planes`` x-z planes (scaled by
    Ny / n_planes), the a5 terms over all modes, the a6-a7 implicit solves
    on ``n_modes`` modes (scaled by M / n_modes) and the a8 mean flow; with
    ``with_filter`` also the filter pass on the same planes.  Returns (seconds per
    substep, seconds per filter pass, wall seconds the sample took, sample sizes).
    """
    import oracle as O
    import synthetic as SY
    st = O.Setup(c["re"], c["Lx"], c["Lz"], c["Nx"], c["Ny"], c["Nz"], c["dt"])
    s0 = SY.turbulent_like(st.y, c["re"], c["Lx"], c["Lz"], c["Nx"], c["Nz"], seed=1)
    S = O.initial_state(st, s0["v"], s0["omega2"], s0["U1"], s0["U3"])
    M = st.Nz * st.nxh
    t_start = t0 = time.perf_counter()
    u1, v, u3, du1, dv, du3 = O.velocities(st, S)
    t_vel = time.perf_counter() - t0
    pl = np.linspace(0, st.Ny - 1, n_planes).astype(int)
    t0 = time.perf_counter()
    om1 = du3[pl] - 1j * st.K3 * v[pl]
    om3 = 1j * st.K1 * v[pl] - du1[pl]
    p = [O.to_physical(st, F) for F in (u1[pl], v[pl], u3[pl], om1, S["omega2"][pl], om3)]
    H1 = p[1] * p[5] - p[2] * p[4]
    H2 = p[2] * p[3] - p[0] * p[5]
    H3 = p[0] * p[4] - p[1] * p[3]
    Hs = [O.to_fourier(st, H) for H in (H1, H2, H3)]
    t_fft = (time.perf_counter() - t0) * st.Ny / n_planes
    H = [np.zeros_like(v) for _ in range(3)]
    for k in range(3):
        H[k][pl] = Hs[k]
    t0 = time.perf_counter()
    Nchi, Nom = O.rhs_terms(st, *H)
    t_rhs = time.perf_counter() - t0
    sel = np.linspace(0, M - 1, n_modes).astype(int)
    sts = copy.copy(st)
    for k in ("K1", "K3", "K2", "keep"):
        setattr(sts, k, getattr(st, k).reshape(1, -1)[:, sel])
    sub = lambda F: F.reshape(st.Ny, 1, M)[:, :, sel]
    Ss = dict(S, v=sub(S["v"]), omega2=sub(S["omega2"]), chi=sub(S["chi"]),
              Nchi_prev=sub(S["Nchi_prev"]), Nom_prev=sub(S["Nom_prev"]))
    t0 = time.perf_counter()
    O.channel.implicit_step(sts, Ss, sub(Nchi), sub(Nom), 0)
    t_imp = (time.perf_counter() - t0) * M / n_modes
    t0 = time.perf_counter()
    O.channel.mean_flow_step(st, S, H[0][:, 0, 0].real, H[2][:, 0, 0].real, 0)
    t_mean = time.perf_counter() - t0
    t_sub = t_vel + t_fft + t_rhs + t_imp + t_mean
    t_filt = 0.0
    if with_filter:
        # the filter pass of a step (Sec. 3.1) on the same planes: G u_i, the products
        # u_i u_j and ubar_i ubar_j, their dealiased projections, tau_ij (scaled by Ny / planes)
        kind, p1, p3 = c["filt"]
        t0 = time.perf_counter()
        G = O.filter_transfer(st, kind, p1, p3)
        u = [u1[pl], v[pl], u3[pl]]
        ub = [G * f for f in u]
        pu = [O.to_physical(st, f) for f in u]
        pb = [O.to_physical(st, f) for f in ub]
        [G * O.to_fourier(st, pu[i] * pu[j]) - O.to_fourier(st, pb[i] * pb[j]) for i, j in O.PAIRS]
        t_filt = (time.perf_counter() - t0) * st.Ny / n_planes + t_vel
    return t_sub, t_filt, time.perf_counter() - t_start, dict(planes=n_planes, modes=n_modes)


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count()


def _anchor_seconds():
    """Best of three whole runs of the oracle on the small workload (after one warm-up)."""
    import oracle as O
    import synthetic as SY
    c = CONFIGS["re180_32x49x32"]
    kind, p1, p3 = c["filt"]
    st = O.Setup(c["re"], c["Lx"], c["Lz"], c["Nx"], c["Ny"], c["Nz"], c["dt"])
    s0 = SY.perturbed_poiseuille(st.y, c["re"], c["Lx"], c["Lz"], c["Nx"], c["Nz"], seed=1, amp=0.1)

    def once():
        t0 = time.perf_counter()
        S = O.run(st, O.initial_state(st, s0["v"], s0["omega2"], s0["U1"], s0["U3"]), c["sub_per_step"])
        O.filter_stresses(st, S, kind, p1, p3)
        return time.perf_counter() - t0

    once()   # warm caches (coefficient systems, FFT plans)
    return min(once() for _ in range(3))


def oracle_anchor_c1():
    """The oracle's full small workload, not extrapolated: Re_tau 180, 32 x 49 x 32,
    10 substeps and the box filter with tau_ij, timed on all host threads and, in a child
    process whose thread pools are limited to one thread, on one."""
    c = CONFIGS["re180_32x49x32"]
    pts = c["Nx"] * c["Ny"] * c["Nz"]
    t_all = _anchor_seconds()
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", "import bench; print(bench._anchor_seconds())"], cwd=ROOT,
                           env=env, capture_output=True, text=True, timeout=600)
        t_one = float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except Exception:
        t_one = None
    val = lambda t: pts * c["sub_per_step"] / t / 1e6 if t else None
    return {"workload": "re180_32x49x32", "substeps": c["sub_per_step"], "filter": "box 50 x 50",
            "seconds_all_threads": t_all, "value_all_threads": val(t_all), "threads": cpu_threads(),
            "seconds_one_thread": t_one, "value_one_thread": val(t_one), "unit": "Mpts*substep/s",
            "timed": "whole run (10 substeps + filter pass), best of 3, not extrapolated"}


def run_reference(args, c, name):
    """The oracle, as it stands, on a bounded sample of each step.

    Each timed step runs the sample of ``oracle_sample_substep_seconds`` (the
    transforms and products on 4 planes, the implicit solves on 512 modes, the
    wall-normal derivatives and mean flow over everything, the filter pass on the
    4 planes); ``ms_per_step`` is the wall time that sample took, and ``value`` the
    throughput of the whole workload implied by scaling each part to its full size
    (``work_per_step_mpts_substep`` = value x the sample's seconds: the share of a
    step's work the sample stands for)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pts = c["Nx"] * c["Ny"] * c["Nz"]
    nsub = c["sub_per_step"]
    full, wall = [], []
    for k in range(args.warmup + args.steps):
        t_sub, t_filt, t_wall, sample = oracle_sample_substep_seconds(c, with_filter=True)
        if k >= args.warmup:
            full.append(nsub * t_sub + t_filt)
            wall.append(t_wall)
    t_step = float(np.median(full))
    t_sample = float(np.median(wall))
    value = pts * nsub / t_step / 1e6
    desc = ("a step of the oracle estimated from a sample: a2-a4 and the filter pass on %d of %d planes, "
            "a6-a7 on %d of %d modes (each scaled to the full size), a1/a5 y-derivatives and a8 over "
            "everything; a step = %d substeps + the filter pass" %
            (sample["planes"], c["Ny"], sample["modes"], c["Nz"] * c["Nx"] // 2, nsub))
    cpu = {"value": value, "unit": "Mpts*substep/s", "cores": cpu_threads(), "kind": "oracle", "sample": desc,
           "cpu_model": cpu_model(), "nproc": os.cpu_count()}
    line = {"impl": "reference", "metric": "DNS Mpts.substep/s", "value": value, "unit": "Mpts*substep/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_sample * 1e3, "ms_per_full_step_estimated": t_step * 1e3,
            "work_per_step_mpts_substep": value * t_sample,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(name, c, "fp64"),
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "Mpts*substep/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_ours(args, c, name):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_1808_06461_b300 as chan
    import synthetic as SY
    precs = {"fp64": chan.CHAN_PREC_FP64, "mixed": chan.CHAN_PREC_MIXED, "f64x": chan.CHAN_PREC_F64X,
             "mixed_df": chan.CHAN_PREC_MIXED_DF}
    stream = torch.cuda.current_stream()
    nsub = c["sub_per_step"]
    kind, p1, p3 = c["filt"]
    pts = c["Nx"] * c["Ny"] * c["Nz"]
    s0 = None
    tuned = {}

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    def ranks_max(x):
        return max_over_ranks(x, dist if world > 1 else None, "cuda")

    def measure(mode, with_clocks):
        """Warm up from the seeded field, snapshot, then time args.steps steps."""
        nonlocal s0
        ch = chan.Channel(c["re"], c["Lx"], c["Lz"], c["Nx"], c["Ny"], c["Nz"], c["dt"], precision=precs[mode],
                          stream=stream.cuda_stream)
        if s0 is None:
            s0 = SY.turbulent_like(ch.grid(), c["re"], c["Lx"], c["Lz"], c["Nx"], c["Nz"], seed=1 + rank)

        def one_step():
            ch.step(nsub)
            ch.filter_stresses(kind, p1, p3, want=False)
            ch.stats()

        ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        # launch shapes for this box (results bitwise unchanged)
        tuned[mode] = ch.tuned_shape() if args.no_autotune else ch.autotune()
        for _ in range(args.warmup):
            one_step()
        snap = ch.get_state()
        snap["stats"] = ch.stats()[0]
        barrier()
        stop, samples = threading.Event(), []
        th = None
        if with_clocks:
            th = threading.Thread(target=clocks_sampler, args=(stop, samples), daemon=True)
            th.start()
        ch.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            one_step()
        e1.record(stream)
        barrier()
        stop.set()
        if th is not None:
            th.join(timeout=10)
        prof = ch.profile_read()
        ch.profile(False)
        ms = ranks_max(e0.elapsed_time(e1))
        return ch, snap, prof, ms, samples

    def roofline(prof, peak64):
        """The dominant kernel's algorithmic flops per step (all its launches) over its
        summed CUDA-event time."""
        dom = max(prof, key=lambda k: prof[k][0])
        dms, dn = prof[dom]
        fl = step_flops(c, nsub).get(dom, 0.0) * args.steps
        achieved = fl / (dms * 1e-3) / 1e12 if dms else 0.0
        return dom, achieved, achieved / peak64

    hbm_peak = measured_peaks().get("hbm_gbs") or 6400.0
    hbm_source = "measured" if measured_peaks().get("hbm_gbs") else "fallback"

    def hbm(prof, mode, step_ms, steps):
        """Algorithmic bytes over time: the dominant kernel's per launch (its bytes per step
        over its launches per step, against its mean CUDA-event launch time) and the whole
        step's (every kernel's bytes per step over the step time)."""
        by = step_bytes(c, mode, nsub)
        dom = max(prof, key=lambda k: prof[k][0])
        dms, dn = prof[dom]
        per_launch = by.get(dom, 0.0) * steps / dn if dn else 0.0
        gbs = per_launch / (dms / dn * 1e-3) / 1e9 if dn else 0.0
        step_gbs = sum(by.values()) / (step_ms * 1e-3) / 1e9
        return {"kernel": dom, "bytes_per_launch": per_launch, "achieved_gbs": gbs, "frac": gbs / hbm_peak,
                "step_bytes": sum(by.values()), "step_achieved_gbs": step_gbs, "step_frac": step_gbs / hbm_peak,
                "bytes_per_pt_substep": sum(by.values()) / (pts * nsub),
                "peak_gbs": hbm_peak, "peak_source": hbm_source + " (MEASURED_PEAKS hbm_gbs, a copy kernel)"
                if hbm_source == "measured" else "fallback 6400 GB/s"}

    main_mode = args.precision
    ch, snap_main, prof, ms, samples = measure(main_mode, True)
    dgemm64 = fp64_peak_tflops(torch)
    peak64 = FP64_PEAK_DERIVED_TFLOPS
    value = replica_throughput(world, args.steps, nsub, pts, ms)

    # ---- end to end through the public API with pinned host buffers
    shape = (c["Ny"], c["Nz"], c["Nx"] // 2)
    n = s0["v"].size
    h2d = 2 * n * 16 + 2 * c["Ny"] * 8
    d2h = (9 * n + 2 * n) * 16 + 2 * c["Ny"] * 8 + (20 * c["Ny"] + 3) * 8
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 3))
    e2e = None
    if e2e_steps:
        pin = lambda n, dt: torch.empty(n, dtype=dt, pin_memory=True).numpy()
        cpin = lambda shp: pin(2 * int(np.prod(shp)), torch.float64).view(np.complex128).reshape(shp)
        hv, ho = cpin(shape), cpin(shape)
        hv[...] = s0["v"]
        ho[...] = s0["omega2"]
        hU1 = pin(c["Ny"], torch.float64); hU1[...] = s0["U1"]
        hU3 = pin(c["Ny"], torch.float64); hU3[...] = s0["U3"]
        # pinned destinations for everything a step reads back (filled in place by the API)
        out_state = dict(v=cpin(shape), omega2=cpin(shape), U1=pin(c["Ny"], torch.float64),
                         U3=pin(c["Ny"], torch.float64))
        out_filt = (cpin((3,) + shape), cpin((6,) + shape))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ch.set_state(hv, ho, hU1, hU3)
            ch.step(nsub)
            ch.filter_stresses(kind, p1, p3, out=out_filt)
            ch.stats()
            ch.get_state(out=out_state)
        barrier()
        e2e = replica_throughput(world, e2e_steps, nsub, pts, ranks_max(time.perf_counter() - t0) * 1e3)
    ch.close()

    dom, achieved, frac = roofline(prof, peak64)
    hbm_main = hbm(prof, main_mode, ms / args.steps, args.steps)
    main_f32 = main_mode in ("mixed", "mixed_df") and dom in ("k_xpass", "k_zinv", "k_zfwd")
    peak_main = FP32_PEAK_DERIVED_TFLOPS if main_f32 else peak64
    frac = achieved / peak_main
    key = (dom, "fp64" if dom in ("k_helm", "k_pre", "k_poisson", "k_nonlin", "k_mean") else main_mode)
    traffic_ncu = (NCU_BYTES_PER_PLANE[key] * c["Ny"]
                   if key in NCU_BYTES_PER_PLANE and c["Nx"] == 384 and c["Nz"] == 384 else None)
    traffic = traffic_ncu if NCU_CURRENT.get(key, False) else None
    launches = int(sum(v[1] for v in prof.values()))
    tot_ms = max(1e-9, sum(x[0] for x in prof.values()))
    kernels = {k: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / tot_ms, 4)}
               for k, v in prof.items() if v[1]}
    peaks = measured_peaks()

    # ---- the other precision modes on the same workload, with their error against FP64
    modes = {}
    if main_mode == "fp64" and not args.no_modes:
        st_main = snap_main["stats"]

        def prof_err(a, b):
            return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

        def rms(stt):
            return np.sqrt(np.maximum(stt[2:5] - np.array([stt[0] ** 2, 0 * stt[0], stt[1] ** 2]), 0.0))

        for mode in ("mixed", "f64x", "mixed_df"):
            chm, snap, profm, msm, _ = measure(mode, False)
            chm.close()
            dm, am, fm = roofline(profm, peak64)
            f32_kernel = mode in ("mixed", "mixed_df") and dm in ("k_xpass", "k_zinv", "k_zfwd")
            peak_m = FP32_PEAK_DERIVED_TFLOPS if f32_kernel else peak64
            fm = am / peak_m
            sm_ = snap["stats"]
            modes[mode] = {
                "value": replica_throughput(world, args.steps, nsub, pts, msm), "ms_per_step": msm / args.steps,
                "roofline": {"kernel": dm, "achieved": am, "frac": fm, "unit": "TFLOP/s", "bound": "alu",
                             "peak": peak_m,
                             "note": ("FP32 algorithmic flops over the FP32 ALU peak derived from unit counts "
                                      "and clocks: 148 SMs x 128 FMA lanes x 2 flop x 2032 MHz" if f32_kernel
                                      else "FP64-equivalent algorithmic flops over the FP64 ALU peak; "
                                      + ("the kernel runs on the FP32 pipe (pair arithmetic), so the ratio can "
                                         "pass 1" if mode == "f64x" and dm in ("k_xpass", "k_zinv", "k_zfwd")
                                         else ("a pair-arithmetic wall-normal kernel (FP32 pipe)" if mode != "mixed"
                                               else "an FP64 wall-normal kernel")))},
                "kernel_shares": {k: round(v[0] / max(1e-9, sum(x[0] for x in profm.values())), 4)
                                  for k, v in profm.items() if v[1]},
                "hbm": hbm(profm, mode, msm / args.steps, args.steps),
                "err_vs_gpu_fp64": {"after_substeps": args.warmup * nsub,
                                "reference": "the FP64 run of this bench (held to the FP64 oracle at 1e-10 "
                                             "relative L2 by the parity tests)",
                                "v_rel_l2": float(np.linalg.norm(snap["v"] - snap_main["v"]) / np.linalg.norm(snap_main["v"])),
                                "omega2_rel_l2": float(np.linalg.norm(snap["omega2"] - snap_main["omega2"]) /
                                                       np.linalg.norm(snap_main["omega2"])),
                                "mean_profile_rel": prof_err(sm_[0], st_main[0]),
                                "rms_profiles_rel": prof_err(rms(sm_), rms(st_main)),
                                "tau_rel": prof_err(sm_[14:20], st_main[14:20])},
                "dtype": {"mixed": "f32 transforms + f64 y-solves",
                          "f64x": "f32x2 transforms and y-sweeps, f64 mean solve",
                          "mixed_df": "f32 transforms + f32x2 y-sweeps, f64 mean solve"}[mode]}
    line = {"metric": "DNS Mpts.substep/s", "value": value, "unit": "Mpts*substep/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "mixed": "f32+f64", "f64x": "f32x2+f64", "mixed_df": "f32+f32x2+f64"}[main_mode],
            "data": "synthetic",
            "config": workload_config(name, c, main_mode, world),
            "launch_shapes": {m: dict(zip(("kb_z", "xthreads", "ytab_global"), v)) for m, v in tuned.items()},
            "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak_main,
                         "unit": "TFLOP/s", "frac": frac, "traffic": traffic,
                         "traffic_source": "ncu dram bytes per plane on 384x33x384, scaled to Ny planes",
                         "traffic_earlier_build": None if traffic is not None else traffic_ncu,
                         "pipe_busy_ncu": NCU_PIPE.get(key),
                         "ncu_counters_current": bool(NCU_CURRENT.get(key, False)),
                         "peak_source": ("FP32 ALU peak derived from unit counts and clocks: 148 SMs x 128 FMA lanes x 2 flop x 2032 MHz"
                                         if main_f32 else
                                         "FP64 ALU peak derived from unit counts and clocks: 148 SMs x 2 DFMA/clk x 2 flop x 2032 MHz"),
                         "dgemm_tflops_measured": dgemm64,
                         "hbm": hbm_main,
                         "hbm_note": ("the FP64 step is FP64-ALU bound on this GPU (FP64 issues at 1/59 of "
                                      "the FP32 rate, 1.2 TFLOP/s against 6.5 TB/s, 0.18 flop/B; the path needs "
                                      "~3 flop/B), so its HBM fraction stays far below the 60 % a bandwidth-bound "
                                      "step would reach" if main_mode == "fp64" else None)},
            "kernels": kernels,
            "gpu_launches": launches,
            "e2e": {"value": e2e, "unit": "Mpts*substep/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "clocks": summarize_clocks(samples)}
    if modes:
        line["modes"] = modes
    if not args.no_serve:
        line["serving"] = run_serving(args, rank)
    if world == 1 and not args.no_configs:
        del ch
        line["configs"] = run_configs(args, chan, SY, torch, precs, stream)
    if rank == 0 and not args.no_cpu_baseline:
        t_sub, t_filt, _, sample = oracle_sample_substep_seconds(c, with_filter=True)
        line["cpu_baseline"] = {"value": pts * nsub / (nsub * t_sub + t_filt) / 1e6, "unit": "Mpts*substep/s",
                                "cores": cpu_threads(), "kind": "oracle", "cpu_model": cpu_model(),
                                "nproc": os.cpu_count(),
                                "sample": "one step (%d substeps + the filter pass) estimated from a2-a4 and the "
                                          "filter on %d of %d planes and a6-a7 on %d of %d modes (scaled), "
                                          "a1/a5/a8 over everything" %
                                          (nsub, sample["planes"], c["Ny"], sample["modes"], c["Nz"] * c["Nx"] // 2),
                                "anchor_c1": oracle_anchor_c1()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_configs(args, chan, SY, torch, precs, stream):
    """The two mixed-precision configurations beside the headline workload.

    Re_tau 1000 (768 x 385 x 768, dt 1e-4): FP64, mixed and mixed with pair sweeps,
    each 500 substeps from the same seeded field and then the sharp filter with
    tau_ij and the statistics, timed with CUDA events; errors of the mean, rms and
    tau_ij profiles against the FP64 run (held to the FP64 oracle at 1e-10 by the
    parity tests), relative to each profile's magnitude and to how far it moved
    from its initial value.
    Re_tau 2000 (1536 x 633 x 1152, dt 5e-5, mixed; the padded 2304-point x
    transform does not fit one CTA in FP64): steps of 20 substeps with the box
    filter of width 100 wall units and the statistics, 1 warm-up step and 2 timed
    steps (40 of the configuration's 200 substeps)."""
    out = {}

    def prof_err(a, b, b0=None):
        d = float(np.abs(a - b).max())
        r = {"rel_to_magnitude": d / max(float(np.abs(b).max()), 1e-300)}
        if b0 is not None:
            r["rel_to_change"] = d / max(float(np.abs(b - b0).max()), 1e-300)
        return r

    def rms(stt):
        return np.sqrt(np.maximum(stt[2:5] - np.array([stt[0] ** 2, 0 * stt[0], stt[1] ** 2]), 0.0))

    def run(cname, modes, nsub, steps, warm):
        c = CONFIGS[cname]
        kind, p1, p3 = c["filt"]
        pts = c["Nx"] * c["Ny"] * c["Nz"]
        res, s0 = {}, None
        for mode in modes:
            torch.cuda.empty_cache()
            ch = chan.Channel(c["re"], c["Lx"], c["Lz"], c["Nx"], c["Ny"], c["Nz"], c["dt"], precision=precs[mode],
                              stream=stream.cuda_stream)
            try:
                if s0 is None:
                    s0 = SY.turbulent_like(ch.grid(), c["re"], c["Lx"], c["Lz"], c["Nx"], c["Nz"], seed=1)
                ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
                ch.filter_stresses(kind, p1, p3, want=False)
                st0 = ch.stats()[0]
                shapes = ch.tuned_shape() if args.no_autotune else ch.autotune()
                ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
                for _ in range(warm):
                    ch.step(nsub)
                    ch.filter_stresses(kind, p1, p3, want=False)
                    ch.stats()
                ch.profile(True)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    ch.step(nsub)
                    ch.filter_stresses(kind, p1, p3, want=False)
                    stt = ch.stats()[0]
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                prof = ch.profile_read()
                ch.profile(False)
                dev_bytes = ch.device_bytes()
            finally:
                ch.close()
            tot = max(1e-9, sum(v[0] for v in prof.values()))
            dom = max(prof, key=lambda k: prof[k][0])
            by = step_bytes(c, mode, nsub)
            dms, dn = prof[dom]
            hb = measured_peaks().get("hbm_gbs") or 6400.0
            f32k = mode in ("mixed", "mixed_df") and dom in ("k_xpass", "k_zinv", "k_zfwd")
            alu_peak = FP32_PEAK_DERIVED_TFLOPS if f32k else FP64_PEAK_DERIVED_TFLOPS
            alu = step_flops(c, nsub).get(dom, 0.0) * steps / (dms * 1e-3) / 1e12 if dms else 0.0
            res[mode] = {"value": pts * nsub * steps / (ms * 1e-3) / 1e6, "unit": "Mpts*substep/s",
                         "ms_per_step": ms / steps, "substeps_timed": nsub * steps, "launch_shapes": shapes,
                         "device_bytes": dev_bytes,
                         "kernel_shares": {k: round(v[0] / tot, 4) for k, v in prof.items() if v[1]},
                         "roofline": {"kernel": dom, "bound": "alu", "achieved_tflops": alu,
                                      "peak_tflops": alu_peak, "frac": alu / alu_peak,
                                      "hbm_kernel_gbs": by.get(dom, 0.0) * steps / dn / (dms / dn * 1e-3) / 1e9,
                                      "hbm_kernel_frac": by.get(dom, 0.0) * steps / (dms * 1e-3) / 1e9 / hb,
                                      "hbm_step_gbs": sum(by.values()) * steps / (ms * 1e-3) / 1e9,
                                      "hbm_step_frac": sum(by.values()) * steps / (ms * 1e-3) / 1e9 / hb,
                                      "hbm_peak_gbs": hb},
                         "_stats": stt, "_stats0": st0}
        if "fp64" in res:
            ref, ref0 = res["fp64"]["_stats"], res["fp64"]["_stats0"]
            for mode in modes:
                if mode == "fp64":
                    continue
                stt = res[mode]["_stats"]
                res[mode]["err_vs_gpu_fp64"] = {
                    "after_substeps": nsub * (warm + steps),
                    "reference": "the FP64 run of the same configuration (held to the FP64 oracle at 1e-10 "
                                 "relative L2 by the parity tests)",
                    "mean_profile": prof_err(stt[0], ref[0], ref0[0]),
                    "rms_profiles": prof_err(rms(stt), rms(ref), rms(ref0)),
                    "tau_profiles": prof_err(stt[14:20], ref[14:20], ref0[14:20]),
                    "uu_profiles": prof_err(stt[2:8], ref[2:8], ref0[2:8])}
        for mode in modes:
            res[mode].pop("_stats")
            res[mode].pop("_stats0")
        return {"config": workload_config(cname, c, "/".join(modes)), "filter_every_substeps": nsub,
                "modes": res}

    out["re1000_768x385x768"] = run("re1000_768x385x768", ("fp64", "mixed", "mixed_df"), 500, 1, 0)
    out["re2000_1536x633x1152"] = run("re2000_1536x633x1152", ("mixed",), 20, 2, 1)
    return out


def run_serving(args, rank):
    """The serving mix: Poisson arrivals (seeded, mean 50 req/s) of minimal-box runs with
    Re_tau in {180, 395, 550}, Nx, Nz in {32, 64, 128}, Ny in {49, 97, 129} and 100-2000
    substeps, served by the continuous-batching loop, in each precision mode."""
    import synthetic as SY
    from paper_1808_06461_b300.serve import Server, channel_factory, poisson_requests

    def ic(r, y):
        return SY.perturbed_poiseuille(y, r.re_tau, r.Lx, r.Lz, r.Nx, r.Nz, seed=r.seed, amp=0.1)

    out = {"requests": args.serve_requests, "rate_per_s": 50.0, "seed": 42, "hbm_budget_gb": 64,
           "max_slots": 16}
    how = {"streams": False, "persistent": "persistent", "packed": True}
    for prec, tag in ((0, "fp64"), (1, "mixed"), (2, "f64x"), (3, "mixed_df")):
        for mode in args.serve_modes.split(","):
            reqs = poisson_requests(args.serve_requests, 50.0, 42 + rank, precision=prec)
            _, m = Server(64 << 30, max_slots=16, factory=channel_factory(ic), packed=how[mode]).run(
                reqs, keep_results=False)
            out[tag + "_" + mode] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in m.items()}
    return out


def run_precision_study(args, c, name):
    """FP64, mixed and double-float runs of ``--precision-study`` substeps from the same seeded
    field; errors of the plane statistics (mean, rms, tau_ij after the filter) against FP64."""
    import torch
    import paper_1808_06461_b300 as chan
    import synthetic as SY
    kind, p1, p3 = c["filt"]
    res, times = {}, {}
    s0 = None
    for tag, prec in (("fp64", chan.CHAN_PREC_FP64), ("mixed", chan.CHAN_PREC_MIXED), ("f64x", chan.CHAN_PREC_F64X),
                      ("mixed_df", chan.CHAN_PREC_MIXED_DF)):
        ch = chan.Channel(c["re"], c["Lx"], c["Lz"], c["Nx"], c["Ny"], c["Nz"], c["dt"], precision=prec,
                          stream=torch.cuda.current_stream().cuda_stream)
        if s0 is None:
            s0 = SY.turbulent_like(ch.grid(), c["re"], c["Lx"], c["Lz"], c["Nx"], c["Nz"], seed=1)
        ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ch.step(args.precision_study)
        ch.sync()
        times[tag] = time.perf_counter() - t0
        ch.filter_stresses(kind, p1, p3, want=False)
        st, utau, ub, f = ch.stats()
        g = ch.get_state()
        res[tag] = dict(stats=st, v=g["v"], om=g["omega2"], utau=utau)
        ch.close()
    ref = res["fp64"]["stats"]

    def rel_prof(a, b):
        return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

    def rms(stt):
        return np.sqrt(np.maximum(stt[2:5] - np.array([stt[0] ** 2, 0 * stt[0], stt[1] ** 2]), 0.0))

    out = {"workload": name, "substeps": args.precision_study, "filter": c["filt"], "seconds": times,
           "mpts_substep_per_s": {k: c["Nx"] * c["Ny"] * c["Nz"] * args.precision_study / v / 1e6 for k, v in times.items()}}
    for tag in ("mixed", "f64x", "mixed_df"):
        st = res[tag]["stats"]
        out[tag + "_vs_fp64"] = {
            "mean_profile_rel": rel_prof(st[0], ref[0]),
            "rms_profiles_rel": rel_prof(rms(st), rms(ref)),
            "tau_profiles_rel": rel_prof(st[14:20], ref[14:20]),
            "uu_profiles_rel": rel_prof(st[2:8], ref[2:8]),
            "v_rel_l2": float(np.linalg.norm(res[tag]["v"] - res["fp64"]["v"]) / np.linalg.norm(res["fp64"]["v"])),
            "utau_rel": abs(res[tag]["utau"] - res["fp64"]["utau"]) / res["fp64"]["utau"]}
    print(json.dumps(out), flush=True)


def run_batch_probe(args):
    """Profiling case of the persistent batch launch: four serving-size runs, one launch of
    12 substeps of each (``--batch-probe``); prints one JSON line with the wall time."""
    import torch
    import synthetic as SY
    import paper_1808_06461_b300 as chan
    prec = {"fp64": 0, "mixed": 1, "f64x": 2, "mixed_df": 3}[args.precision]
    runs = []
    for (nx, ny, nz, re) in ((32, 49, 32, 180.0), (64, 97, 64, 395.0), (128, 129, 128, 550.0), (64, 49, 128, 395.0)):
        ch = chan.Channel(re, math.pi, math.pi / 2, nx, ny, nz, 2e-4, precision=prec)
        s0 = SY.perturbed_poiseuille(ch.grid(), re, math.pi, math.pi / 2, nx, nz, seed=nx + ny, amp=0.1)
        ch.set_state(s0["v"], s0["omega2"], s0["U1"], s0["U3"])
        runs.append(ch)
    b = chan.ChannelBatch(runs, persistent=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(12)
    b.status()
    t = time.perf_counter() - t0
    pts = sum(ch.Nx * ch.Ny * ch.Nz for ch in runs)
    b.close()
    print(json.dumps({"probe": "persistent batch", "runs": 4, "substeps": 12, "points": pts, "seconds": t}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed", "f64x", "mixed_df"], default="fp64")
    ap.add_argument("--no-modes", action="store_true", help="skip the mixed / double-float runs")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-mix run")
    ap.add_argument("--serve-requests", type=int, default=96)
    ap.add_argument("--serve-modes", default="streams,persistent",
                    help="comma-separated serving issue modes: streams (per-run streams), persistent "
                         "(one work-list launch per RK3 step of all runs), packed (one launch per kernel)")
    ap.add_argument("--precision-study", type=int, default=0,
                    help="run FP64 / mixed / double-float for this many substeps and report profile errors")
    ap.add_argument("--config", choices=sorted(CONFIGS), default=DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the Re 1000 and Re 2000 mixed-precision configuration runs")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes (profiling runs)")
    ap.add_argument("--batch-probe", action="store_true",
                    help="profiling case of the persistent batch launch (four serving-size runs, 12 substeps)")
    args = ap.parse_args()
    c = CONFIGS[args.config]
    if args.batch_probe:
        run_batch_probe(args)
    elif args.precision_study:
        run_precision_study(args, c, args.config)
    elif args.impl == "reference":
        run_reference(args, c, args.config)
    else:
        run_ours(args, c, args.config)


if __name__ == "__main__":
    main()
