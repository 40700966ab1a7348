"""Benchmark of the nested-grid lattice Boltzmann hot path on GB300.

Headline workload: 256^3 periodic decaying turbulence (random-phase
solenoidal field, E(k) ~ k^4 exp(-2 (k/k0)^2), k0 = 4, u_rms = 0.04,
nu = 1e-4), D3Q27 factorized cascaded collision, FP32 storage.  One "step" is
one coarse time step (one fused stream-collide launch over all 16.8 M cells
in a CUDA graph).  Metric: MLUPS (million lattice-cell updates per second),
with the HBM-roofline fraction of the stream-collide kernel at 216 algorithmic
bytes per FP32 D3Q27 update (27 values read + 27 written).

Also reported ("variants"): FP16 storage and D3Q19 MRT-LES on the same grid,
the 2-level round-jet grid (coarse 384x192x192, fine cylinder of radius 24
coarse cells), the FP64-storage run, and the velocity error of FP32 / FP16
storage against the FP64 run after a fixed number of steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per GPU, launched by torchrun): the
update has no exchange step on one GPU, so there is no collective; value is
the whole-job MLUPS (all replicas' updates / the max time over ranks).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline, FP32/FP16-storage vs FP64 at stated error"
N_GRID = 256
NU = 1e-4
OMEGA = 1.0 / (3.0 * NU + 0.5)
BYTES_PER_UPDATE = {("d3q27", "f32"): 216, ("d3q27", "f16"): 108, ("d3q27", "f64"): 432,
                    ("d3q19", "f32"): 152, ("d3q19", "f16"): 76, ("d3q19", "f64"): 304}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "update_kernel_traffic.txt")
KERNEL_SOURCES = ["paper_1206_0389_gb300/csrc/update.cuh", "paper_1206_0389_gb300/csrc/pair.cuh",
                  "paper_1206_0389_gb300/csrc/collide.cuh",
                  "paper_1206_0389_gb300/csrc/lattice.cuh"]


# ----------------------------------------------------------------- distributed helpers
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value, device=None):
    """Max of a float over ranks (identity on one rank)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value, device=None):
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_mlups(updates_all_ranks, max_ms):
    return updates_all_ranks / (max_ms * 1e-3) / 1e6


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        self.proc.wait()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------- roofline inputs
def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic_per_update(model, storage):
    """DRAM bytes per cell update from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    kv = {}
    for line in open(TRAFFIC_FILE):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_sha") != kernel_sha():
        return None
    key = "bytes_per_update_%s_%s" % (model, storage)
    return float(kv[key]) if key in kv else None


# ----------------------------------------------------------------- our arm
def run_uniform(lbm, torch, model, storage, field, steps, warmup, stream, sampler=None):
    """Time `steps` coarse steps of the 256^3 periodic grid; returns a dict."""
    nb = (N_GRID // 8,) * 3
    ctx = lbm.lbm_create(model, storage, nb, True, [], OMEGA, 0.1 if model == "d3q19" else 0.0,
                         stream.cuda_stream)
    rho, u = field
    lbm.lbm_init_equilibrium(ctx, 0, rho, u)
    lbm.lbm_step(ctx, warmup)
    lbm.lbm_sync(ctx)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.start()
    e0.record(stream)
    lbm.lbm_step(ctx, steps)
    e1.record(stream)
    e1.synchronize()
    clocks = sampler.stop() if sampler else None
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # profiled pass: per-launch CUDA events around each kernel on the same stream
    lbm.lbm_set_profiling(ctx, True)
    prof_steps = max(5, min(steps, 50))
    lbm.lbm_step(ctx, prof_steps)
    pms, pn = lbm.lbm_get_profile(ctx)
    lbm.lbm_set_profiling(ctx, False)
    threads, minb, ctas = lbm.lbm_get_tuning(ctx)
    out = dict(ctx=ctx, ms=ms, clocks=clocks, kernel_ms=pms[0] / max(pn[0], 1),
               launches_per_step=int(pn.sum()) // prof_steps, tuning=(threads, minb, ctas),
               cells=N_GRID ** 3)
    return out


def roofline(model, storage, kernel_ms, cells):
    peak, src = measured_peak()
    bpu = BYTES_PER_UPDATE[(model, storage)]
    achieved = bpu * cells / (kernel_ms * 1e-3) / 1e9
    t = ncu_traffic_per_update(model, storage)
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": src,
            "traffic": None if t is None else round(t * cells),
            "algorithmic_bytes_per_launch": bpu * cells}


def velocity_error(lbm, ctx, ref_u):
    _, u = lbm.lbm_macroscopic(ctx, 0)
    return float(np.sqrt(((u - ref_u) ** 2).sum() / (ref_u ** 2).sum()))


def run_jet(lbm, torch, model, steps, warmup, stream, walls=0, slip=0, paper_tank=False):
    """2-level jet (coarse 384x192x192, fine cylinder of radius 24 coarse
    cells); walls/slip put it in a tank (y/z wall faces, free-slip subset).
    paper_tank adds the rest of the paper's setup: the pressure outlet (the
    refinement then stops one block before it) and the nozzle, a cylinder
    of diameter 16 from x = 8 to 48 (coarse cells) on the fine level whose
    cap emits the jet."""
    import synth
    flags, centre = synth.jet_two_level()
    outlet, nozzle = 0, None
    if paper_tank:
        flags = [flags[0].copy()]
        flags[0][:, :, -1] = False
        outlet, nozzle = 1, (centre[0], centre[1], 8.0, 8.0, 48.0)
    kw = dict(walls=walls, slip=slip, outlet=outlet, nozzle=nozzle)
    nu_c = 0.05 * 16 / 1e4
    ctx = lbm.lbm_create(model, "f32", (48, 24, 24), False, flags, 1.0 / (3 * nu_c + 0.5),
                         0.18 if model == "d3q19" else 0.0, stream.cuda_stream, **kw)
    lbm.lbm_set_inflow(ctx, centre[0], centre[1], 16.0, 0.05, 0.01, 389)
    info = lbm.lbm_plan((48, 24, 24), False, flags, model, "f32", **kw)
    lbm.lbm_step(ctx, warmup)
    lbm.lbm_sync(ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lbm.lbm_step(ctx, steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    lbm.lbm_set_profiling(ctx, True)
    lbm.lbm_step(ctx, 3)
    pms, pn = lbm.lbm_get_profile(ctx)
    lbm.lbm_destroy(ctx)
    upd = info.active_updates_per_coarse_step
    peak, _ = measured_peak()
    bpu = BYTES_PER_UPDATE[(model, "f32")]
    return {"mlups": round(upd / (ms * 1e-3) / 1e6, 1), "ms_per_coarse_step": round(ms, 4),
            "active_updates_per_coarse_step": int(upd),
            "frac_of_hbm_roofline": round(bpu * upd / (ms * 1e-3) / 1e9 / peak, 4),
            "profile_ms_per_coarse_step": {k: round(float(v) / 3, 4) for k, v in
                                           zip(["update", "c2f", "f2c", "bc", "other"], pms)},
            "launches_per_coarse_step": int(pn.sum()) // 3}


def run_sharded(lbm, torch, field, steps, warmup, stream, nparts):
    """The headline grid (256^3 D3Q27 FP32) cut into nparts parts on this
    one GPU: each coarse step runs the halo exchange of every cut (pack,
    device-to-device copy, unpack) and then each part's step, every part on
    a stream of its own."""
    nb = (N_GRID // 8,) * 3
    sh = lbm.lbm_shard_create("d3q27", "f32", nb, True, [], OMEGA, 0.0, nparts, stream.cuda_stream)
    lbm.lbm_shard_init_equilibrium(sh, 0, *field)
    lbm.lbm_shard_step(sh, warmup)
    lbm.lbm_shard_sync(sh)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lbm.lbm_shard_step(sh, steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    cuts = [lbm.lbm_shard_part(sh, p)[1] for p in range(nparts)] + [nb[0]]
    halo = lbm.lbm_shard_halo_bytes(sh)
    lbm.lbm_shard_destroy(sh)
    return {"parts": nparts, "cuts_level0_columns": cuts, "ms_per_step": round(ms, 4),
            "mlups": round(N_GRID ** 3 / (ms * 1e-3) / 1e6, 1), "halo_bytes_per_step": halo,
            "what": "all parts on one GPU, each on its own stream; the exchange is pack + device-to-device "
                    "copy + unpack per cut"}


def run_jet3(lbm, torch, storage, steps, warmup, stream):
    """3-level jet at the paper's scale (coarse 512x256x256, nozzle D = 32,
    rings along the shear layer, 40.09 M active cells), D3Q27 FCLB."""
    import synth
    flags, centre = synth.jet_paper_scale()
    nu_c = 0.05 * 32 / 1e4
    ctx = lbm.lbm_create("d3q27", storage, (64, 32, 32), False, flags, 1.0 / (3 * nu_c + 0.5), 0.0,
                         stream.cuda_stream)
    lbm.lbm_set_inflow(ctx, centre[0], centre[1], 32.0, 0.05, 0.01, 5120)
    info = lbm.lbm_plan((64, 32, 32), False, flags, "d3q27", storage)
    lbm.lbm_step(ctx, warmup)
    lbm.lbm_sync(ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lbm.lbm_step(ctx, steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    lbm.lbm_set_profiling(ctx, True)
    lbm.lbm_step(ctx, 2)
    pms, pn = lbm.lbm_get_profile(ctx)
    lbm.lbm_set_profiling(ctx, False)
    m = lbm.lbm_mass_momentum(ctx)
    # time-averaged centreline velocity over the next 50 coarse steps (not
    # timed; the paper's evaluation quantity, reported, not gated): the axis
    # lies on level 0 (the refined rings start at r = 8)
    lbm.lbm_stats_reset(ctx)
    for _ in range(50):
        lbm.lbm_step(ctx, 1)
        lbm.lbm_stats_accumulate(ctx)
    mean, var, nsamp = lbm.lbm_stats_get(ctx, 0)
    jy, jz = int(centre[0]) - 1, int(centre[1]) - 1
    axis_ux = mean[1, jz:jz + 2, jy:jy + 2, :].mean(axis=(0, 1))
    axis_var = var[0, jz:jz + 2, jy:jy + 2, :].mean(axis=(0, 1))
    centreline = {"%g" % xd: round(float(axis_ux[int(xd * 32)]) / 0.05, 5) for xd in (0, 0.25, 0.5, 1, 2)}
    intensity = {"%g" % xd: round(float(np.sqrt(max(axis_var[int(xd * 32)], 0.0))) / 0.05, 5)
                 for xd in (0, 0.25, 0.5)}
    # ring profiles over all levels (area-weighted) on cross-sections near
    # the nozzle and the jet quantities of Section 3.3 from them
    stations = (0.1, 0.25)
    pm, pv, pc = lbm.lbm_stats_radial(ctx, -1, centre[0], centre[1], 1.0, 40, [xd * 32 for xd in stations])
    profile = {}
    for s, xd in enumerate(stations):
        um, be, ti, a, c = lbm.lbm_jet_fit(pm[s], pv[s], pc[s], 1.0)
        fin = lambda v, nd: round(v, nd) if np.isfinite(v) else None      # JSON has no NaN
        profile["%g" % xd] = {"u_m_over_u_in": fin(um / 0.05, 5), "half_width_over_D": fin(be / 32, 5),
                              "turbulence_intensity": fin(ti, 5), "gauss_a": fin(a, 4), "gauss_c": fin(c, 4)}
    total_steps = warmup + steps + 2 + 50
    lbm.lbm_destroy(ctx)
    upd = info.active_updates_per_coarse_step
    peak, _ = measured_peak()
    bpu = BYTES_PER_UPDATE[("d3q27", storage)]
    return {"mlups": round(upd / (ms * 1e-3) / 1e6, 1), "ms_per_coarse_step": round(ms, 4),
            "active_cells": [int(info.active_cells[l]) for l in range(3)],
            "active_updates_per_coarse_step": int(upd), "steps": steps,
            "frac_of_hbm_roofline": round(bpu * upd / (ms * 1e-3) / 1e9 / peak, 4),
            "profile_ms_per_coarse_step": {k: round(float(v) / 2, 4) for k, v in
                                           zip(["update", "c2f", "f2c", "bc", "other"], pms)},
            "launches_per_coarse_step": int(pn.sum()) // 2, "final_momentum_x": float(m[1]),
            "centreline_mean_ux_over_u_in_by_x_over_D": centreline,
            "centreline_rms_ux_over_u_in_by_x_over_D": intensity,
            "jet_profile_by_x_over_D": profile,
            "statistics_window": "coarse steps %d-%d after start from rest (%d samples)" % (
                total_steps - 50 + 1, total_steps, nsamp)}


def run_adjoint(lbm, torch, stream, T=256, every=16, N=96):
    """Adjoint of the forced FCLB update (96^3, FP32, T = 256): device time
    of the T forward steps vs the recording forward and the backward sweep,
    for checkpoints every `every` steps (recompute + adjoint) and for the
    library's own choice (every state kept when it fits: no recompute)."""
    import synth
    omega = 1.0 / (3 * 0.005 + 0.5)
    rho, u = synth.spectrum_field(N, seed=4096)
    F = synth.random_force((N, N, N), 4096, sigma=1e-6)
    ctx = lbm.lbm_create("d3q27", "f32", (N // 8,) * 3, True, [], omega, 0.0, stream.cuda_stream)
    lbm.lbm_init_equilibrium(ctx, 0, rho, u)
    lbm.lbm_set_force(ctx, F)
    f0 = lbm.lbm_get_state(ctx, 0)
    lbm.lbm_step(ctx, 3)
    lbm.lbm_sync(ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lbm.lbm_step(ctx, T)
    e1.record(stream)
    e1.synchronize()
    fwd_ms = e0.elapsed_time(e1)
    lam = np.zeros((27, N, N, N))
    c = N // 2
    lam[:, c - 8:c + 8, c - 8:c + 8, c - 8:c + 8] = 1e-3
    modes = {}
    for ev in (every, 0):
        lbm.lbm_set_state(ctx, 0, f0)
        lbm.lbm_adjoint_forward(ctx, T, ev)       # allocation outside the timed pass
        lbm.lbm_set_state(ctx, 0, f0)
        lbm.lbm_sync(ctx)
        e0.record(stream)
        lbm.lbm_adjoint_forward(ctx, T, ev)
        e1.record(stream)
        e1.synchronize()
        ckfwd_ms = e0.elapsed_time(e1)
        used = lbm.lbm_adjoint_generation(ctx)[1]
        lbm.lbm_set_profiling(ctx, True)
        lbm.lbm_adjoint_backward(ctx, lam)
        pms, _ = lbm.lbm_get_profile(ctx)
        lbm.lbm_set_profiling(ctx, False)
        sweep_ms = float(pms[4])
        modes["auto" if ev == 0 else "every_%d" % ev] = {
            "checkpoint_every": used, "recording_forward_ms": round(ckfwd_ms, 3),
            "backward_sweep_ms": round(sweep_ms, 3), "backward_over_forward": round(sweep_ms / fwd_ms, 3),
            "adjoint_total_over_forward": round((ckfwd_ms + sweep_ms) / fwd_ms, 3)}
    lbm.lbm_destroy(ctx)
    return {"grid": "%d^3" % N, "T": T, "forward_ms": round(fwd_ms, 3), "modes": modes,
            "adjoint_total_over_forward": modes["auto"]["adjoint_total_over_forward"]}


# D3Q27 velocities in the library's order (for the FP16 bound's constant)
_E27 = np.array([[0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, 1, -1, -1, 1, -1],
                 [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, 1, -1, 1, -1, -1],
                 [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, 1, -1, -1, -1]])
_W27 = np.array([{0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}[int((_E27[:, i] ** 2).sum())] for i in range(27)])


def fp16_injection_rms(f_cells):
    """rms over sampled cells (f_cells [n][27], unshifted) of
    I = sqrt(sum_i |e_i|^2 g_i^2), g_i = f_i - w_i: one step of FP16 storage
    rounds each g_i by at most 2^-11 |g_i|, so it moves the momentum of a
    cell by at most 2^-11 I times a factor near one.  The stated bound after
    N steps is B = sqrt(N) 2^-11 rms(I at t = 0) / rms(u after N steps)."""
    g = f_cells - _W27[None, :]
    inj = np.sqrt(((_E27 ** 2).sum(0)[None, :] * g * g).sum(1))
    return float(np.sqrt((inj ** 2).mean()))


def energy_spectrum(u, kmax):
    """Shell-summed kinetic energy spectrum E(k), k = 1..kmax, of a periodic
    field u [3][N][N][N] (E summed over |k| in [k - 1/2, k + 1/2))."""
    N = u.shape[1]
    uk = np.fft.rfftn(u, axes=(1, 2, 3)) / N ** 3
    e = 0.5 * (np.abs(uk) ** 2).sum(0)
    e[..., 1:(N + 1) // 2] *= 2.0          # the conjugate half of the rfft
    kk = np.fft.fftfreq(N, d=1.0 / N)
    kr = np.arange(uk.shape[-1])
    kmag = np.sqrt(kk[:, None, None] ** 2 + kk[None, :, None] ** 2 + kr[None, None, :] ** 2)
    shell = np.rint(kmag).astype(np.int64)
    E = np.bincount(shell.ravel(), weights=e.ravel(), minlength=kmax + 1)
    return E[1:kmax + 1]


def run_config2_diagnostics(lbm, torch, field, stream, steps=2000, every=100):
    """The 256^3 decaying-turbulence field (D3Q27 FCLB) run in FP64, FP32
    and FP16 storage side by side for `steps` steps: kinetic energy and the
    velocity relative L2 divergence of FP32/FP16 from FP64 every `every`
    steps, energy spectra at t = 0, steps/2, steps, and the FP16 bound
    beside its measured value.  Not gated: the flow is chaotic, so rounding
    differences grow exponentially and pass any rounding bound within about
    a thousand steps (the bound is for non-chaotic flows, see
    run_fp16_bound_laminar and the GPU tests)."""
    cells = N_GRID ** 3
    rho, u0 = field
    ctxs = {}
    for st in ("f64", "f32", "f16"):
        ctxs[st] = lbm.lbm_create("d3q27", st, (N_GRID // 8,) * 3, True, [], OMEGA, 0.0, stream.cuda_stream)
        lbm.lbm_init_equilibrium(ctxs[st], 0, rho, u0)
    rng = np.random.default_rng(2000)
    sample = rng.choice(cells, size=65536, replace=False).astype(np.int64)
    I0 = fp16_injection_rms(lbm.lbm_get_cells(ctxs["f64"], 0, sample).reshape(-1, 27))
    urms = {}
    t0 = time.perf_counter()
    energy = {st: [] for st in ctxs}
    div = {"f32": [], "f16": []}
    spectra = {}
    kmax = 64
    for t in range(0, steps + 1, every):
        if t > 0:
            for c in ctxs.values():
                lbm.lbm_step(c, every)
        us = {}
        for st, c in ctxs.items():
            _, us[st] = lbm.lbm_macroscopic(c, 0)
            energy[st].append(float(0.5 * (us[st] ** 2).sum(0).mean()))
        ref = us["f64"]
        nref = float(np.sqrt((ref ** 2).sum()))
        urms[t] = nref / math.sqrt(cells)
        for st in div:
            div[st].append(float(np.sqrt(((us[st] - ref) ** 2).sum())) / nref)
        if t in (0, steps // 2, steps):
            spectra[str(t)] = {st: [float("%.4g" % v) for v in energy_spectrum(us[st], kmax)] for st in ctxs}
        del us, ref
    for c in ctxs.values():
        lbm.lbm_destroy(c)
    ts = list(range(0, steps + 1, every))
    bound = {str(n): math.sqrt(n) * 2.0 ** -11 * I0 / urms[n] for n in (100, 1000, 2000) if n in urms}
    measured = {str(n): div["f16"][ts.index(n)] for n in (100, 1000, 2000) if n in ts}
    return {"grid": "256^3 periodic", "model": "d3q27", "steps": steps, "every": every,
            "t": ts, "kinetic_energy": {k: [float("%.6g" % v) for v in e] for k, e in energy.items()},
            "velocity_rel_l2_vs_f64": {k: [float("%.4g" % v) for v in d] for k, d in div.items()},
            "spectra_k1_to_%d" % kmax: spectra,
            "fp16_bound": {"form": "sqrt(N) * 2^-11 * rms(I at t = 0) / rms(u_N), I = sqrt(sum_i |e_i|^2 "
                                   "(f_i - w_i)^2) (65,536 sampled cells)",
                           "bound": {k: float("%.4g" % v) for k, v in bound.items()},
                           "measured": {k: float("%.4g" % v) for k, v in measured.items()}},
            "host_s": round(time.perf_counter() - t0, 1)}


def run_fp16_bound_laminar(lbm, torch, stream, steps=1000):
    """The FP16 bound on a non-chaotic flow of the same grid: a 256^3
    Taylor-Green vortex (u0 = 0.04, D3Q27 FCLB, the decaying-turbulence
    viscosity) in FP16 and FP32 storage against an FP64 run after `steps`
    steps, beside the stated bound (fp16_injection_rms)."""
    import synth
    cells = N_GRID ** 3
    rho, u = synth.taylor_green_3d(N_GRID, 0.04)
    out = {}
    ctxs = {}
    for st in ("f64", "f32", "f16"):
        ctxs[st] = lbm.lbm_create("d3q27", st, (N_GRID // 8,) * 3, True, [], OMEGA, 0.0, stream.cuda_stream)
        lbm.lbm_init_equilibrium(ctxs[st], 0, rho, u)
    sample = np.random.default_rng(1000).choice(cells, size=65536, replace=False).astype(np.int64)
    I0 = fp16_injection_rms(lbm.lbm_get_cells(ctxs["f64"], 0, sample).reshape(-1, 27))
    for c in ctxs.values():
        lbm.lbm_step(c, steps)
    _, ref = lbm.lbm_macroscopic(ctxs["f64"], 0)
    nref = float(np.sqrt((ref ** 2).sum()))
    urms = nref / math.sqrt(cells)
    for st in ("f32", "f16"):
        _, ug = lbm.lbm_macroscopic(ctxs[st], 0)
        out[st] = float("%.4g" % (float(np.sqrt(((ug - ref) ** 2).sum())) / nref))
        del ug
    for c in ctxs.values():
        lbm.lbm_destroy(c)
    return {"case": "256^3 Taylor-Green vortex, u0 = 0.04, D3Q27 FCLB, nu = 1e-4, %d steps vs FP64 storage" % steps,
            "form": "sqrt(N) * 2^-11 * rms(I at t = 0) / rms(u_N), I = sqrt(sum_i |e_i|^2 (f_i - w_i)^2)",
            "bound": float("%.4g" % (math.sqrt(steps) * 2.0 ** -11 * I0 / urms)),
            "measured_f16": out["f16"], "measured_f32": out["f32"]}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def oracle_mlups(model, N, threads, steps=1):
    """The FP64 oracle as it stands on an N^3 periodic sample of the
    decaying-turbulence workload: MLUPS of `steps` timed steps with
    `threads` torch threads (after one untimed step below 64^3, where the
    first step's set-up would weigh; from 64^3 a step takes seconds)."""
    import torch
    import synth
    from oracle.solver import NestedSolver
    prev = torch.get_num_threads()
    torch.set_num_threads(threads)
    try:
        s = NestedSolver(model, (N // 8,) * 3, periodic_x=True, omega=OMEGA, cs=0.1 if model == "d3q19" else 0.0)
        rho, u = synth.spectrum_field(N, seed=1206)
        s.init_equilibrium(0, torch.from_numpy(rho), torch.from_numpy(u))
        if N < 64:
            s.step(1)
        t0 = time.perf_counter()
        s.step(steps)
        dt = time.perf_counter() - t0
        used = torch.get_num_threads()
    finally:
        torch.set_num_threads(prev)
    return N ** 3 * steps / dt / 1e6, dt, used


def cpu_baseline(full=False, budget_s=45.0):
    """The FP64 oracle on the host cores, per model, size and thread count:
    64^3 with all cores and with one thread, 128^3 with all cores (and one
    thread with full=True), one timed step each; a run stops adding cases
    once the budget of timed seconds is spent (the rest are listed as
    skipped).  The headline value is D3Q27 at 64^3 on all cores."""
    import torch
    cores = torch.get_num_threads()
    cases = [("d3q27", 64, cores), ("d3q27", 64, 1), ("d3q19", 64, cores), ("d3q19", 64, 1),
             ("d3q27", 128, cores), ("d3q19", 128, cores)]
    if full:
        cases += [("d3q27", 128, 1), ("d3q19", 128, 1)]
    per, spent = [], 0.0
    for model, N, th in cases:
        if spent > budget_s:
            per.append({"model": model, "grid": "%d^3" % N, "threads": th, "skipped": "time budget"})
            continue
        v, dt, used = oracle_mlups(model, N, th)
        spent += dt
        per.append({"model": model, "grid": "%d^3" % N, "threads": used, "mlups": round(v, 5),
                    "step_s": round(dt, 2)})
    head = per[0]
    return {"value": head["mlups"], "unit": "MLUPS", "cores": head["threads"], "kind": "oracle",
            "cpu_model": cpu_model(), "host_cores": os.cpu_count(),
            "sample": "FP64 oracle (plain PyTorch CPU ops), one timed step per case on periodic samples of "
                      "the k^4-spectrum workload; value = D3Q27 FCLB at 64^3 on all cores",
            "per_case": per}


def ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    import synth
    import __graft_entry__
    __graft_entry__.build() if not os.path.exists(
        os.path.join(ROOT, "paper_1206_0389_gb300", "liblbm.so")) else None
    from paper_1206_0389_gb300 import lbm
    stream = torch.cuda.Stream()
    field = synth.spectrum_field(N_GRID, seed=1206 + rank)
    K, W = args.steps, args.warmup

    if args.kernel_only and args.variant.startswith(("jet2s_", "jet2t_", "jet2p_", "jet3s_", "jet3p_")):
        # jets for profiling the interface and boundary kernels:
        # jet2s = 2 levels (coarse 192x96x96, fine cylinder of radius 12);
        # jet2t = jet2s in a tank (no-slip sides and bottom, free-slip top);
        # jet2p = the paper's tank at that size: walls, pressure outlet and the
        # nozzle (diameter 8, x = 8..24) on the fine level (refinement radius 20);
        # jet3s = the 3-level jet at half the paper's scale (coarse
        # 256x128x128, D = 16, 1.8 GB in FP32); jet3p = the paper-scale
        # 3-level jet (11.3 GB in FP32: launch lists only, no full captures)
        kind, model, storage = args.variant.split("_")
        walls, slip = (15, 8) if kind in ("jet2t", "jet2p") else (0, 0)
        outlet, nozzle = 0, None
        if kind in ("jet2s", "jet2t"):
            nb, D = (24, 12, 12), 8.0
            flags, centre = synth.jet_two_level(*nb, radius=12.0)
        elif kind == "jet2p":
            nb, D = (24, 12, 12), 8.0
            flags, centre = synth.jet_two_level(*nb, radius=20.0)
            flags = [flags[0].copy()]
            flags[0][:, :, -1] = False
            outlet, nozzle = 1, (centre[0], centre[1], 4.0, 8.0, 24.0)
        elif kind == "jet3p":
            nb, D = (64, 32, 32), 32.0
            flags, centre = synth.jet_paper_scale()
        else:
            nb, D = (32, 16, 16), 16.0
            flags, centre = synth.jet_three_level(*nb, r1=(4.0, 16.0), r2=(6.0, 12.0), x1=(0, 96), x2=(0, 48))
        ctx = lbm.lbm_create(model, storage, nb, False, flags, 1.0 / (3 * 8e-5 + 0.5),
                             0.18 if model == "d3q19" else 0.0, stream.cuda_stream, walls=walls, slip=slip,
                             outlet=outlet, nozzle=nozzle)
        lbm.lbm_set_inflow(ctx, centre[0], centre[1], D, 0.05, 0.01, 389)
        lbm.lbm_step(ctx, W)
        # the coarse-step graphs (level-0 update beside the fine levels),
        # then the same steps as sequential launches timed per kind
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lbm.lbm_step(ctx, K)
        e1.record(stream)
        e1.synchronize()
        graph_ms = e0.elapsed_time(e1) / K
        lbm.lbm_set_profiling(ctx, True)
        lbm.lbm_step(ctx, K)
        pms, pn = lbm.lbm_get_profile(ctx)
        lbm.lbm_destroy(ctx)
        if rank == 0:
            print(json.dumps({"kernel_only": True, "variant": args.variant,
                              "graph_ms_per_coarse_step": round(graph_ms, 4),
                              "ms_per_coarse_step": {k: float(v) / K for k, v in
                                                     zip(["update", "c2f", "f2c", "bc", "other"], pms)},
                              "launches": [int(x) for x in pn]}), flush=True)
        return
    if args.kernel_only and args.variant.startswith("sharded_"):
        # the headline grid in P block-sharded parts (sharded_<P>)
        r = run_sharded(lbm, torch, field, K, W, stream, int(args.variant.split("_")[1]))
        if rank == 0:
            print(json.dumps({"kernel_only": True, "variant": args.variant, **r}), flush=True)
        return
    if args.kernel_only and args.variant.startswith("audit_"):
        # the float64 mass/momentum audit (k_reduce) on an N^3 periodic grid
        _, model, storage = args.variant.split("_")
        N = args.grid
        fld = synth.spectrum_field(N, seed=1206)
        ctx = lbm.lbm_create(model, storage, (N // 8,) * 3, True, [], OMEGA, 0.0, stream.cuda_stream)
        lbm.lbm_init_equilibrium(ctx, 0, *fld)
        for _ in range(W):
            lbm.lbm_mass_momentum(ctx)
        t0 = time.perf_counter()
        for _ in range(K):
            m = lbm.lbm_mass_momentum(ctx)
        dt = (time.perf_counter() - t0) / K
        lbm.lbm_destroy(ctx)
        if rank == 0:
            print(json.dumps({"kernel_only": True, "variant": args.variant, "grid": N,
                              "ms_per_audit_call": dt * 1e3, "sums": [float(v) for v in m]}), flush=True)
        return
    if args.kernel_only and args.variant == "adjoint":
        # the adjoint pipeline at 96^3 with a short horizon (profiling k_adjoint)
        r = run_adjoint(lbm, torch, stream, T=32, every=8)
        if rank == 0:
            print(json.dumps({"kernel_only": True, "variant": "adjoint", **r}), flush=True)
        return
    if args.kernel_only:
        model, storage = args.variant.split("_")
        r = run_uniform(lbm, torch, model, storage, field, K, W, stream)
        lbm.lbm_destroy(r["ctx"])
        if rank == 0:
            print(json.dumps({"kernel_only": True, "ms_per_step": r["ms"] / K,
                              "kernel_ms": r["kernel_ms"], "tuning": r["tuning"]}), flush=True)
        return

    # headline: D3Q27 FCLB FP32
    barrier(dist)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    head = run_uniform(lbm, torch, "d3q27", "f32", field, K, W, stream, sampler)
    barrier(dist)
    ms_max = max_over_ranks(dist, head["ms"], device="cuda")
    updates_all = sum_over_ranks(dist, head["cells"] * K, device="cuda")
    value = whole_job_mlups(updates_all, ms_max)
    roof = roofline("d3q27", "f32", head["kernel_ms"], head["cells"])
    ctx = head["ctx"]
    lbm.lbm_destroy(ctx)

    # end to end through the C ABI with host buffers: upload the initial field
    # from pinned memory, K steps each followed by the float64 audit read
    # back to the host, then the macroscopic field back to pinned memory
    rho_h = torch.from_numpy(field[0]).pin_memory()
    u_h = torch.from_numpy(field[1]).pin_memory()
    rho_o = torch.empty_like(rho_h).pin_memory()
    u_o = torch.empty_like(u_h).pin_memory()
    ctx = lbm.lbm_create("d3q27", "f32", (32, 32, 32), True, [], OMEGA, 0.0, stream.cuda_stream)
    lbm.lbm_step(ctx, 1)
    lbm.lbm_sync(ctx)
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lib = lbm.load()
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    st = lib.lbm_init_equilibrium(ctx.h, 0, ctypes.cast(rho_h.data_ptr(), dp), ctypes.cast(u_h.data_ptr(), dp))
    assert st == 0, lbm.lbm_last_error(ctx)
    audit = np.empty(4)
    for _ in range(K):
        lbm.lbm_step(ctx, 1)
        st = lib.lbm_mass_momentum(ctx.h, audit.ctypes.data_as(dp))
        assert st == 0, lbm.lbm_last_error(ctx)
    st = lib.lbm_macroscopic(ctx.h, 0, ctypes.cast(rho_o.data_ptr(), dp), ctypes.cast(u_o.data_ptr(), dp))
    assert st == 0, lbm.lbm_last_error(ctx)
    e2e_ms = (time.perf_counter() - t0) * 1e3
    lbm.lbm_destroy(ctx)
    barrier(dist)
    e2e_max = max_over_ranks(dist, e2e_ms, device="cuda")
    cells = N_GRID ** 3
    h2d = 4 * cells * 8
    d2h = 4 * cells * 8 + 32 * K
    e2e = {"value": round(whole_job_mlups(updates_all, e2e_max), 1), "unit": "MLUPS",
           "h2d_bytes_per_step": int(h2d / K), "d2h_bytes_per_step": int(d2h / K),
           "what": "init from pinned host rho/u + K x (step + float64 audit to host) + rho/u to pinned host"}

    variants = {}
    errors = {}
    if not args.quick:
        # FP64 storage throughput (its storage error is in config2_diagnostics)
        E = 100
        ref = run_uniform(lbm, torch, "d3q27", "f64", field, E, 0, stream)
        variants["d3q27_f64"] = {"mlups": round(cells * E / (ref["ms"] * 1e-3) / 1e6, 1),
                                 "roofline_frac": roofline("d3q27", "f64", ref["kernel_ms"], cells)["frac"]}
        lbm.lbm_destroy(ref["ctx"])
        for model, storage in (("d3q27", "f16"), ("d3q19", "f32"), ("d3q19", "f16")):
            r = run_uniform(lbm, torch, model, storage, field, K, W, stream)
            rf = roofline(model, storage, r["kernel_ms"], cells)
            variants["%s_%s" % (model, storage)] = {
                "mlups": round(cells * K / (r["ms"] * 1e-3) / 1e6, 1), "roofline_frac": rf["frac"],
                "achieved_gbs": rf["achieved"], "tuning": list(r["tuning"])}
            lbm.lbm_destroy(r["ctx"])
        errors["fp16_bound_nonchaotic"] = run_fp16_bound_laminar(lbm, torch, stream)
        errors["config2_diagnostics"] = run_config2_diagnostics(lbm, torch, field, stream)
        for model in ("d3q27", "d3q19"):
            variants["jet_2level_%s_f32" % model] = run_jet(lbm, torch, model, max(10, K // 4), 3, stream)
        # the same jet in a tank: no-slip side walls and bottom, free-slip top
        variants["jet_2level_tank_d3q27_f32"] = run_jet(lbm, torch, "d3q27", max(10, K // 4), 3, stream,
                                                        walls=15, slip=8)
        # and the paper's whole tank: plus the pressure outlet and the nozzle
        variants["jet_2level_paper_tank_d3q27_f32"] = run_jet(lbm, torch, "d3q27", max(10, K // 4), 3, stream,
                                                              walls=15, slip=8, paper_tank=True)
        for storage in ("f32", "f16"):
            variants["jet_3level_d3q27_%s" % storage] = run_jet3(lbm, torch, storage, max(20, K // 4), 3, stream)
        variants["adjoint_d3q27_f32"] = run_adjoint(lbm, torch, stream)
        for P in (2, 4):
            variants["sharded_d3q27_f32_%dparts" % P] = run_sharded(lbm, torch, field, max(20, K // 4), 3, stream, P)

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": round(ms_max / K, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "256^3 periodic decaying turbulence, D3Q27 FCLB, FP32 storage "
                               "(k^4 spectrum, k0=4, u_rms=0.04, nu=1e-4)",
                   "cells": cells, "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (1.81 GB per distribution buffer)",
                   "launch": {"threads": head["tuning"][0], "min_ctas_per_sm": head["tuning"][1],
                              "ctas": head["tuning"][2]}},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": head["launches_per_step"] * K,
        "clocks": head["clocks"],
        "kernel_ms": round(head["kernel_ms"], 4),
        "variants": variants,
        "storage_error": errors,
    }
    if rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline(full=args.cpu_baseline_full)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def reference(args):
    """The oracle timed on the host cores on the same metric (bounded sample)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import torch
    import synth
    from oracle.solver import NestedSolver
    s = NestedSolver("d3q27", (2, 2, 2), periodic_x=True, omega=OMEGA)
    rho, u = synth.spectrum_field(16, seed=1206)
    s.init_equilibrium(0, torch.from_numpy(rho), torch.from_numpy(u))
    for _ in range(args.warmup):
        s.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(1)
    dt = time.perf_counter() - t0
    v = 16 ** 3 * args.steps / dt / 1e6
    cb = {"value": round(v, 6), "unit": "MLUPS", "cores": torch.get_num_threads(), "kind": "oracle",
          "sample": "D3Q27 FCLB FP64 oracle, 16^3 periodic sample of the 256^3 k^4-spectrum workload, "
                    "%d steps" % args.steps}
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "256^3 periodic decaying turbulence, D3Q27 FCLB (16^3 sample on the host)"},
            "cpu_baseline": cb,
            "e2e": {"value": round(v, 6), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--quick", action="store_true", help="headline only (no variants)")
    ap.add_argument("--grid", type=int, default=256, help="for --kernel-only audit_*: N of the N^3 grid")
    ap.add_argument("--cpu-baseline-full", action="store_true",
                    help="also time the oracle single-threaded at 128^3 (minutes)")
    ap.add_argument("--kernel-only", action="store_true",
                    help="only the stream-collide steps of one variant (for ncu captures)")
    ap.add_argument("--variant", default="d3q27_f32",
                    help="for --kernel-only: model_storage (e.g. d3q19_f16), jet2s_/jet2t_/jet2p_/jet3s_/jet3p_"
                         "model_storage, audit_model_storage, adjoint, or sharded_<parts>")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
