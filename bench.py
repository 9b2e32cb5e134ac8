"""Throughput of the fused f+g time step (MLUPS) and its HBM roofline.

Default workload: 4096 x 1024 heated-wall boiling layout (bounce-back walls
top and bottom, 32-cell hot spot at T/Tc = 0.95 on the bottom wall, bulk at
T/Tc = 0.8, liquid below y = 768 and vapour above, body force 1e-5 down),
FP32 population storage -- the "FP32 plain" form every other form is
compared against. A step is one fused launch: pull streaming, density and
pair force, EOS, f and g collision, store, and the FP64 conservation
reduction. The state (2 x 302 MB) is larger than L2, so no flush is needed
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision f64|f32|f16s|bf16s] [--rounding 1|0]

Studies (one JSON line each, no timing contract):
  --batch-study STEPS      the 256-case sweep against the Maxwell densities
  --precision-study STEPS  the storage formats (16-bit with stochastic and
                           nearest rounding) side by side against FP64
  --laplace-study STEPS    eight static droplets in one periodic 512 x 512 box
                           at T/Tc 0.7, 0.8, 0.9: pressure jump against 1/R,
                           spurious currents, FP32 against FP64
  --stefan-study, --droplet-study N   the open heated sides (Eq. 20, D^2 law)
  --droplet-pair-study N   the paper's evaporating droplet pair scaled to N x N

Under torchrun (N > 1) every rank runs an independent replica of the
workload (the method has no exchange between independent cases); the value
is the sum of lattice updates over all ranks divided by the slowest rank's
time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY = 4096, 1024
Y_INT = 768


def set_size(nx, ny):
    global NX, NY
    NX, NY = nx, ny


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def hbm_peak(peaks):
    for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs", "hbm"):
        if k in peaks:
            v = peaks[k]
            return float(v["value"] if isinstance(v, dict) else v)
    return 6800.0


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


METRIC = "MLUPS of the fused f+g step (FP32 plain)"

# DRAM bytes (read + write) of one k_step launch on this workload, from one
# ncu capture (profiles/k_step_f32_4096x1024_full.md), valid only for the
# kernel sources it was taken on: any change to them makes it null.
STEP_TRAFFIC = {"bytes_per_launch": (309391616 + 255389184 + 308886528 + 253282560) // 2,
                "sources_sha256": "22adc04600794184e7f2dc0308ed44331d9bf8cfaa462689084fc037aff67e11"}
STEP_SOURCES = ["lbm_step.cu", "lbm_device.cuh", "lbm_internal.h", "lbm_ptx.cuh"]


def step_traffic():
    """The captured traffic per launch, or None once the kernel changed."""
    import hashlib
    h = hashlib.sha256()
    root = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2106_01557_gb300", "csrc")
    for f in STEP_SOURCES:
        with open(os.path.join(root, f), "rb") as fh:
            h.update(fh.read())
    return STEP_TRAFFIC["bytes_per_launch"] if h.hexdigest() == STEP_TRAFFIC["sources_sha256"] else None


def slowest_rank_ms(ms, world, device):
    """The whole-job clock: the largest of the ranks' timed durations
    (every rank has passed the same barriers around its timed region)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank, world, ms_step):
    """Lattice updates of all ranks per second (weak scaling: each rank
    advances its own replica of the workload)."""
    return nodes_per_rank * world / (ms_step * 1e-3) / 1e6


def boiling_case(lbm, nx, ny, precision, stream_ptr=None, **overrides):
    from paper_2106_01557_gb300 import inputs
    x0 = inputs.hot_spot_x0(nx, 32, seed=3)
    cfg = lbm.default_config(nx, ny, precision=precision, walls=1, accel_y=-1e-5, Tr_bottom=0.8,
                             Tr_hot=0.95, hot_x0=x0, hot_len=32, Tr_top=0.0, **overrides)
    if stream_ptr is not None:
        cfg.stream = stream_ptr
    lat = lbm.Lattice(cfg)
    p = lat.params()
    rho = inputs.layer(nx, ny, p["rho_v"], p["rho_l"], Y_INT * ny / 1024.0, 4.0)
    T = np.full((ny, nx), p["T0"])
    z = np.zeros((ny, nx))
    return lat, (rho, z, z.copy(), T)


def run_ours(args, rank, world):
    import torch
    from paper_2106_01557_gb300 import lbm

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    prec = args.precision
    lat, fields = boiling_case(lbm, NX, NY, prec, stream_ptr=stream.cuda_stream, rounding=args.rounding)
    lat.set_fields(*fields)
    nodes = NX * NY
    bytes_step = lat.bytes_per_step()

    for _ in range(args.warmup):
        lat.step(1)
    lat.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        time.sleep(0.3)
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
        ev1.synchronize()
        time.sleep(0.2)
    lat.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    stats = lat.step_stats()
    ms = slowest_rank_ms(ms, world, "cuda")
    ms_step = ms / args.steps
    mlups = whole_job_mlups(nodes, world, ms_step)

    # end to end through the public API with host buffers: set fields from
    # pinned host memory, run K steps, read the moments back into pinned
    # host memory (the caller's buffers, filled in place)
    rho, ux, uy, T = (torch.from_numpy(a).pin_memory() for a in fields)
    outs = {k: torch.empty((NY, NX), dtype=torch.float64).pin_memory().numpy() for k in ("rho", "ux", "uy", "T")}
    lat.set_fields(rho.numpy(), ux.numpy(), uy.numpy(), T.numpy())   # untimed: first-touch of the pages
    lat.moments(out=outs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.set_fields(rho.numpy(), ux.numpy(), uy.numpy(), T.numpy())
    lat.step(args.steps)
    lat.moments(out=outs)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": nodes * world * args.steps / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": 4 * 8 * nodes / args.steps, "d2h_bytes_per_step": 4 * 8 * nodes / args.steps,
           "what": "lbm_set_fields(host) + lbm_step(K) + lbm_moments(host) per K steps"}

    variants = {}
    if rank == 0 and not args.no_variants:
        variants = precision_variants(lbm, torch, args.variant_steps)
        variants["batch_f16s"] = batch_variant(lbm, torch, 100)
        if args.surrogate_iters:
            from paper_2106_01557_gb300 import surrogate as sur_mod
            variants["surrogate"] = sur_mod.study(iters=args.surrogate_iters)
            # the same study at longer jumps: the network's cost stays, the LB's grows with K
            scan = []
            for K in [int(k) for k in args.surrogate_ks.split(",") if k]:
                st = sur_mod.study(iters=args.surrogate_iters, K=K)
                ro = st["rollout"]
                scan.append({"K": K, "holdout_gain_vs_persistence": st["holdout_gain_vs_persistence"],
                             "accepted": ro.get("accepted"), "fallbacks": ro.get("fallbacks"),
                             "speedup_vs_lb": ro.get("speedup_vs_lb"),
                             "ms_per_jump_network_only": ro.get("ms_per_jump_network_only"),
                             "ms_per_jump_lb_steps": ro.get("ms_per_jump_lb_steps"),
                             "err_vs_lb": ro.get("err_vs_lb"), "error": ro.get("error")})
            variants["surrogate_k_scan"] = scan
    return {"ms_step": ms_step, "mlups": mlups, "bytes_step": bytes_step, "clocks": clk.summary(),
            "e2e": e2e, "stats": stats.tolist(), "variants": variants}


def precision_variants(lbm, torch, nsteps):
    """The other storage formats on the same workload: MLUPS over `nsteps`
    steps, and the per-field error of FP32 / FP16S / BF16S against the FP64
    run (the FP64 GPU path matches the FP64 oracle to 1e-12): max |x - x64| /
    max |x64| for rho and T, max |u - u64| / c for velocity."""
    out, ref = {}, None
    for prec in ("f64", "f32", "f16s", "bf16s"):
        stream = torch.cuda.Stream()
        lat, fields = boiling_case(lbm, NX, NY, prec, stream_ptr=stream.cuda_stream)
        lat.set_fields(*fields)
        lat.step(3)
        lat.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lat.step(nsteps - 3)
        ev1.record(stream)
        ev1.synchronize()
        lat.synchronize()
        ms = ev0.elapsed_time(ev1) / (nsteps - 3)
        m = lat.moments()
        c = lat.params()["c"]
        rec = {"mlups": NX * NY / (ms * 1e-3) / 1e6, "ms_per_step": ms,
               "bytes_per_lu": lat.bytes_per_step() / (NX * NY)}
        if prec == "f64":
            ref = m
        else:
            rec["err_vs_f64_after_steps"] = nsteps
            rec["err_rho"] = float(np.abs(m["rho"] - ref["rho"]).max() / np.abs(ref["rho"]).max())
            rec["err_T"] = float(np.abs(m["T"] - ref["T"]).max() / np.abs(ref["T"]).max())
            rec["err_u_over_c"] = float(max(np.abs(m["ux"] - ref["ux"]).max(), np.abs(m["uy"] - ref["uy"]).max()) / c)
        out[prec] = rec
        lat.close()
    base = out["f32"]["mlups"]
    for prec in out:
        out[prec]["speedup_vs_f32"] = out[prec]["mlups"] / base
    return out


# The sweep's relaxation rates of g: the paper leaves sigma_eps and sigma_p
# free; 1.4 and 1.8 keep both bulk phases linearly stable at rest down to
# T/Tc = 0.65 (the default rates only to 0.75) and pass every oracle pin.
SWEEP_RATES = dict(sig_eps=1.4, sig_p=1.8)
SWEEP_TR_LO = 0.65


def batch_cases_fields(lbm, ncases, seed, precision, stream_ptr):
    """The heterogeneous sweep: ncases periodic boxes, sides log-uniform in
    [64, 512] (multiples of 8), one droplet of radius U[8, 0.3 min(nx, ny)]
    at the centre, T/Tc uniform in [0.65, 0.95], tanh edge of width 4, with
    the g rates sigma_eps = 1.4, sigma_p = 1.8 (below T/Tc = 0.65 the bulk
    liquid of the model is linearly unstable even with these; the benchmark
    list's range starts at 0.6)."""
    from paper_2106_01557_gb300 import inputs
    cases = inputs.batch_cases(ncases, seed, tr_lo=SWEEP_TR_LO)
    cfgs = []
    for c in cases:
        cfg = lbm.default_config(c["nx"], c["ny"], precision=precision, Tr0=c["Tr"], **SWEEP_RATES)
        if stream_ptr is not None:
            cfg.stream = stream_ptr
        cfgs.append(cfg)
    return cases, cfgs


def batch_variant(lbm, torch, steps, ncases=256, seed=4):
    """Batched FP16-storage sweep in one persistent launch per step (autotuned)
    against the same cases run one by one on the plain FP32 path."""
    from paper_2106_01557_gb300 import inputs
    stream = torch.cuda.Stream()
    cases, cfgs = batch_cases_fields(lbm, ncases, seed, "f16s", stream.cuda_stream)
    b = lbm.Batch(cfgs)
    fields = []
    for i, c in enumerate(cases):
        p = b.params(i)
        rho = inputs.droplets(c["nx"], c["ny"], p["rho_v"], p["rho_l"], [(c["nx"] / 2, c["ny"] / 2)], [c["R"]], 4.0)
        T = np.full_like(rho, p["T0"])
        z = np.zeros_like(rho)
        fields.append((rho, z, z, T))
        b.set_fields(i, *fields[-1])
    choice, ms = b.autotune(5)
    b.step(20)
    b.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.step(steps)
    ev1.record(stream)
    ev1.synchronize()
    b.synchronize()
    ms_step = ev0.elapsed_time(ev1) / steps
    nodes = b.nodes
    out = {"cases": ncases, "nodes": nodes, "mlups": nodes / (ms_step * 1e-3) / 1e6, "ms_per_step": ms_step,
           "bytes_per_lu": b.bytes_per_step() / nodes,
           "autotune": {"tile_shape": ["64x32", "32x16"][choice[0]], "order": lbm.Batch.ORDERS[choice[1]],
                        "ms_per_step_candidates": [round(float(x), 4) for x in ms]}}
    b.close()
    # the same cases, each on its own plain FP32 handle, stepped one after another
    lats = []
    for cfg, fl in zip(batch_cases_fields(lbm, ncases, seed, "f32", stream.cuda_stream)[1], fields):
        lat = lbm.Lattice(cfg)
        lat.set_fields(*fl)
        lats.append(lat)
    per = 20
    for lat in lats:
        lat.step(per)
    torch.cuda.synchronize()
    ev0.record(stream)
    for lat in lats:
        lat.step(per)
    ev1.record(stream)
    ev1.synchronize()
    ms_plain = ev0.elapsed_time(ev1) / per
    for lat in lats:
        lat.close()
    out["plain_f32_one_by_one_mlups"] = nodes / (ms_plain * 1e-3) / 1e6
    out["speedup_vs_plain_f32_one_by_one"] = ms_plain / ms_step
    return out


def batch_study(steps, ncases=256, seed=4, precision="f16s"):
    """The heterogeneous sweep run for `steps` steps (FP16 storage, FP32
    math): per case, the droplet-centre (liquid) and corner (vapour) densities
    against the coexistence densities across a curved interface (Laplace's
    law): equal chemical potentials with the pressure jump sigma(T) / R, R the
    droplet's equimolar radius sqrt(A / pi), A = sum (rho - rho_vb) /
    (rho_lb - rho_vb) from the measured bulk densities, sigma from
    square-gradient theory, each bulk at its own measured temperature (all
    from the library's host solvers). The flat (Maxwell) reference is
    reported beside it. A case whose droplet has evaporated (centre density
    below the mean of the two Maxwell densities) is reported and left out of
    the 1% statistic."""
    import torch
    from paper_2106_01557_gb300 import inputs, lbm
    stream = torch.cuda.Stream()
    cases, cfgs = batch_cases_fields(lbm, ncases, seed, precision, stream.cuda_stream)
    b = lbm.Batch(cfgs)
    for i, c in enumerate(cases):
        p = b.params(i)
        rho = inputs.droplets(c["nx"], c["ny"], p["rho_v"], p["rho_l"], [(c["nx"] / 2, c["ny"] / 2)], [c["R"]], 4.0)
        z = np.zeros_like(rho)
        b.set_fields(i, rho, z, z, np.full_like(rho, p["T0"]))
    b.autotune(5)
    t0 = time.perf_counter()
    b.step(steps)
    diverged = set()
    try:
        b.synchronize()
    except lbm.LbmError:
        # a case whose density went non-finite or non-positive: the cases are
        # independent, so the others are still valid; the record of the last
        # step names the diverged ones
        diverged = {i for i in range(ncases) if b.step_stats(i)[6] > 0}
    wall = time.perf_counter() - t0
    rows, ok, ok_flat, evap = [], 0, 0, 0
    for i, c in enumerate(cases):
        if i in diverged:
            rows.append({"nx": c["nx"], "ny": c["ny"], "R0": round(c["R"], 2), "Tr": round(c["Tr"], 4),
                         "diverged": True, "evaporated": False})
            continue
        m = b.moments(i)
        p = b.params(i)
        cy, cx = c["ny"] // 2, c["nx"] // 2
        rl, Tl = m["rho"][cy, cx], m["T"][cy, cx]
        rv, Tv = m["rho"][0, 0], m["T"][0, 0]
        Mv = lbm.maxwell(cfgs[i], Tv / p["Tc"])[0]
        Ml = lbm.maxwell(cfgs[i], Tl / p["Tc"])[1]
        gone = rl < 0.5 * (Mv + Ml)
        row = {"nx": c["nx"], "ny": c["ny"], "R0": round(c["R"], 2), "Tr": round(c["Tr"], 4),
               "Tr_vapour": round(float(Tv / p["Tc"]), 5), "Tr_liquid": round(float(Tl / p["Tc"]), 5),
               "err_rho_v_flat": rv / Mv - 1, "err_rho_l_flat": rl / Ml - 1, "evaporated": bool(gone)}
        if gone:
            evap += 1
        else:
            area = float(((m["rho"] - rv) / (rl - rv)).sum())
            R = math.sqrt(max(area, 1e-12) / math.pi)
            Lv = lbm.coexistence(cfgs[i], Tv / p["Tc"], lbm.surface_tension(cfgs[i], Tv / p["Tc"]) / R)[0]
            Ll = lbm.coexistence(cfgs[i], Tl / p["Tc"], lbm.surface_tension(cfgs[i], Tl / p["Tc"]) / R)[1]
            ev, el = rv / Lv - 1, rl / Ll - 1
            row.update({"R_equimolar": round(R, 3), "err_rho_v": ev, "err_rho_l": el})
            ok += abs(ev) < 0.01 and abs(el) < 0.01
            ok_flat += abs(row["err_rho_v_flat"]) < 0.01 and abs(row["err_rho_l_flat"]) < 0.01
        rows.append(row)
    b.close()
    kept = [r for r in rows if not r["evaporated"] and not r.get("diverged")]
    med = lambda k: float(np.median([r[k] for r in kept])) if kept else None
    return {"metric": "batched sweep coexistence vs the Laplace-shifted equilibrium", "steps": steps,
            "cases": ncases, "storage": precision, "rates": SWEEP_RATES, "tr_range": [SWEEP_TR_LO, 0.95],
            "wall_s": wall, "evaporated": evap, "diverged": len(diverged),
            "diverged_cases": [rows[i] for i in sorted(diverged)],
            "within_1pct": int(ok), "within_1pct_of_flat_maxwell": int(ok_flat), "of_kept": len(kept),
            "median_err": {"rho_v": med("err_rho_v"), "rho_l": med("err_rho_l"),
                           "rho_v_flat": med("err_rho_v_flat"), "rho_l_flat": med("err_rho_l_flat")},
            "max_abs_err_kept": max((max(abs(r["err_rho_v"]), abs(r["err_rho_l"])) for r in kept), default=None),
            "per_case": rows}


def droplet_study(n=1024, D0=256.0, Tr1=0.85, cv=11.2, precision="f32", samples=24, max_steps=40_000_000,
                  every=None):
    """A droplet of diameter D0 evaporating in an n x n box heated from all
    four sides (open sides at T_r 0.85 and the liquid's saturation
    pressure; the droplet at T_r 0.8; c_v = 11.2 R gives Ste = 0.005 with the
    model's latent heat), as in the paper's D^2-law run (1024^2, D0 = 256).
    Reports (D / D0)^2 against t* = alpha_v t / D0^2 (D from the liquid area,
    D = 2 sqrt(A / pi), A = sum (rho - rho_v) / (rho_l - rho_v)), the slope of
    a straight-line fit over 0.8 > (D/D0)^2 > 0.2 with its coefficient of
    determination, and the quasi-steady conduction rate of a cylinder in a
    square box, d(D^2)/dt = -8 alpha_v Ste / ln(1.08 (n / 2) / R), at the
    fit's mid-point."""
    from paper_2106_01557_gb300 import inputs, lbm
    cfg = lbm.default_config(n, n, precision=precision, walls=1, open_sides=15, Tr_open=Tr1, c_v=cv)
    lat = lbm.Lattice(cfg)
    p = lat.params()
    rho = inputs.droplets(n, n, p["rho_v"], p["rho_l"], [(n / 2 - 0.5, n / 2 - 0.5)], [D0 / 2], 4.0)
    lat.set_fields(rho, 0 * rho, 0 * rho, 0 * rho + p["T0"])
    h_lv = p["a"] * (p["rho_l"] - p["rho_v"]) + p["p_s"] * (1 / p["rho_v"] - 1 / p["rho_l"])
    T1 = Tr1 * p["Tc"]
    ste = p["rho_v"] * p["cv"] * (T1 - p["T0"]) / (p["rho_l"] * h_lv)
    alpha_v = (4 + 3 * cfg.gamma1 + 2 * cfg.gamma2) / 6 * p["Cref"] * p["c"] * cfg.tau_j_v / (p["rho_v"] * p["cv"])
    # quasi-steady lifetime estimate sets the sampling interval
    life = D0 * D0 * math.log(1.08 * n / D0) / (8 * alpha_v * ste) / p["dt"]
    every = every or max(1000, int(life / samples))
    rows, done, t_start = [], 0, time.perf_counter()
    while done < max_steps:
        m = lat.moments()
        r = m["rho"]
        area = float(((r - p["rho_v"]) / (p["rho_l"] - p["rho_v"])).clip(0, None).sum())
        D = 2 * math.sqrt(area / math.pi)
        t = done * p["dt"]
        rows.append({"steps": done, "t_star": alpha_v * t / D0 ** 2, "D2": (D / D0) ** 2,
                     "T_centre_over_Tc": float(m["T"][n // 2, n // 2] / p["Tc"])})
        if (D / D0) ** 2 < 0.05 or r.max() < 0.5 * (p["rho_v"] + p["rho_l"]):
            break
        lat.step(every)
        done += every
    lat.close()
    pts = [(q["t_star"], q["D2"]) for q in rows if 0.2 < q["D2"] < 0.8]
    fit = None
    if len(pts) >= 3:
        x = np.array([a for a, _ in pts])
        y = np.array([b for _, b in pts])
        A = np.vstack([x, np.ones_like(x)]).T
        (k, c), res, *_ = np.linalg.lstsq(A, y, rcond=None)
        ss = float(((y - (k * x + c)) ** 2).sum())
        r2 = 1 - ss / float(((y - y.mean()) ** 2).sum())
        Rm = 0.5 * D0 * math.sqrt(0.5)
        qs = 8 * ste / math.log(1.08 * (n / 2) / Rm)      # -d(D/D0)^2 / dt* at (D/D0)^2 = 0.5
        fit = {"slope": float(k), "intercept": float(c), "r2": r2, "quasi_steady_slope_at_half": -qs,
               "slope_over_quasi_steady": float(-k / qs)}
    return {"metric": "droplet evaporation (D^2 law) on the GPU path", "lattice": [n, n], "D0": D0,
            "storage": precision, "Ste": ste, "alpha_v": alpha_v, "steps_per_sample": every,
            "wall_s": time.perf_counter() - t_start, "fit": fit, "samples": rows}


def droplet_pair_study(n=1024, stes=(0.005, 0.05, 0.5), Tr1=0.85, precision="f32", samples=40,
                       max_steps=60_000_000, report=None):
    """The paper's large-small droplet pair (diameters 160 and 96, centres 256
    apart on 1024 x 1024, everything scaled by n / 1024) heated from all four
    sides (open sides at T_r 0.85 and the liquid's saturation pressure, the
    droplets at T_r 0.8), for each Stefan number in `stes`: Ste is set
    through c_v (Ste = rho_v c_v (T_1 - T_0) / (rho_l h_lv) with the model's
    latent heat h_lv); C_ref = rho_v c_v follows c_v, so the vapour's thermal
    diffusivity alpha_v does not change and a larger Ste evaporates faster.
    Samples, against t* = alpha_v t / D0^2 (D0 = 128 n / 1024): the total
    liquid volume V / V0 (V0 = pi D0^2 / 4; V = sum (rho - rho_v) /
    (rho_l - rho_v) over the liquid components grown by 4 nodes), the number
    of droplets (connected components of rho above the mean of the two
    coexistence densities, at least 20 nodes), the distance between the two
    largest droplets' centroids, and max |u| / c. Each case runs at most four
    times the quasi-steady lifetime estimate of the large droplet; `report`
    (if given) receives each case's result as it completes."""
    from scipy import ndimage
    from paper_2106_01557_gb300 import inputs, lbm
    s = n / 1024.0
    DL, DS, sep, D0 = 160 * s, 96 * s, 256 * s, 128 * s
    probe = lbm.Lattice(lbm.default_config(n, n, precision=precision, walls=1, open_sides=15, Tr_open=Tr1))
    p1 = probe.params()
    probe.close()
    h_lv = p1["a"] * (p1["rho_l"] - p1["rho_v"]) + p1["p_s"] * (1 / p1["rho_v"] - 1 / p1["rho_l"])
    out = []
    for ste in stes:
        cv = ste * p1["rho_l"] * h_lv / (p1["rho_v"] * (Tr1 * p1["Tc"] - p1["T0"]))
        cfg = lbm.default_config(n, n, precision=precision, walls=1, open_sides=15, Tr_open=Tr1, c_v=cv)
        lat = lbm.Lattice(cfg)
        p = lat.params()
        cy = n / 2 - 0.5
        rho = inputs.droplets(n, n, p["rho_v"], p["rho_l"], [(n / 2 - sep / 2, cy), (n / 2 + sep / 2, cy)],
                              [DL / 2, DS / 2], 4.0)
        lat.set_fields(rho, 0 * rho, 0 * rho, 0 * rho + p["T0"])
        alpha_v = (4 + 3 * cfg.gamma1 + 2 * cfg.gamma2) / 6 * p["Cref"] * p["c"] * cfg.tau_j_v / (p["rho_v"] * p["cv"])
        ste_m = p["rho_v"] * p["cv"] * (Tr1 * p["Tc"] - p["T0"]) / (p["rho_l"] * h_lv)
        life = DL * DL * math.log(1.08 * n / DL) / (8 * alpha_v * ste_m) / p["dt"]
        every = max(200, int(life / samples))
        cap = min(max_steps, int(4 * life))
        mid = 0.5 * (p["rho_v"] + p["rho_l"])
        rows, done, err, t0 = [], 0, None, time.perf_counter()
        while done < cap:
            m = lat.moments()
            r = m["rho"]
            lab, nl = ndimage.label(r > mid)
            sizes = ndimage.sum(np.ones_like(r), lab, range(1, nl + 1)) if nl else []
            comps = [k + 1 for k in range(nl) if sizes[k] >= 20]
            phi = ((r - p["rho_v"]) / (p["rho_l"] - p["rho_v"]))
            grown = ndimage.binary_dilation(np.isin(lab, comps), iterations=4) if comps else np.zeros_like(r, bool)
            V = float(phi[grown].sum())
            vols = sorted(((float(phi[lab == k].sum()), k) for k in comps), reverse=True)
            dist = None
            if len(vols) >= 2:
                ca = ndimage.center_of_mass(phi.clip(0, None), lab, [vols[0][1], vols[1][1]])
                dist = float(math.hypot(ca[0][0] - ca[1][0], ca[0][1] - ca[1][1]))
            rows.append({"steps": done, "t_star": alpha_v * done * p["dt"] / D0 ** 2, "V_over_V0": V / (math.pi * D0 * D0 / 4),
                         "droplets": len(comps), "distance": dist,
                         "max_u_over_c": float(np.hypot(m["ux"], m["uy"]).max() / p["c"])})
            if not comps or V < 0.02 * math.pi * D0 * D0 / 4:
                break
            lat.step(every)
            try:
                lat.synchronize()
            except lbm.LbmError as e:
                err = str(e)[:120]
                break
            done += every
        lat.close()
        d = [q["distance"] for q in rows if q["distance"] is not None]
        two = [q for q in rows if q["droplets"] >= 2]
        # coalescence: one droplet left, the pair having come closer than at the
        # start, and no loss of volume across the transition (when the small
        # droplet evaporates instead, its volume is gone)
        merged = None
        for a, b in zip(rows, rows[1:]):
            if (a["droplets"] >= 2 and b["droplets"] == 1 and a["distance"] is not None and d
                    and a["distance"] < d[0] and b["V_over_V0"] >= 0.97 * a["V_over_V0"]):
                merged = b["t_star"]
                break
        out.append({"Ste": ste_m, "c_v": cv, "alpha_v": alpha_v, "steps_per_sample": every, "steps": done,
                    "lifetime_estimate_steps": life, "wall_s": time.perf_counter() - t0, "error": err,
                    "distance_initial": d[0] if d else None, "distance_min": min(d) if d else None,
                    "distance_max": max(d) if d else None, "distance_last_pair": two[-1]["distance"] if two else None,
                    "coalesced_at_t_star": merged, "V_over_V0_max": max(q["V_over_V0"] for q in rows),
                    "t_star_end": rows[-1]["t_star"], "samples": rows})
        if report:
            report(out[-1])
    return {"metric": "large-small droplet pair evaporating, heated from all sides", "lattice": [n, n],
            "diameters": [DL, DS], "centre_distance": sep, "D0": D0, "storage": precision, "results": out}


def _periodic_labels(mask):
    """Connected components of a periodic 2-D mask (4-connectivity, labels
    joined across both edges); 0 outside the mask."""
    from scipy import ndimage
    lab, n = ndimage.label(mask)
    parent = list(range(n + 1))

    def root(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for a, b in list(zip(lab[:, 0], lab[:, -1])) + list(zip(lab[0, :], lab[-1, :])):
        if a and b:
            ra, rb = root(a), root(b)
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    m = np.array([root(a) for a in range(n + 1)])
    out = m[lab]
    ids = [k for k in np.unique(out) if k]
    return out, ids


def laplace_study(steps=50_000, n=512, ndrop=8, seed=2, temps=(0.7, 0.8, 0.9), precisions=("f64", "f32")):
    """Static droplets in one periodic box: ndrop droplets of radius
    U[20, 80] (seeded, centres by rejection sampling with a periodic gap of
    R1 + R2 + 8), tanh edges of width 4 between the Maxwell densities, u = 0,
    uniform T, for `steps` steps at each T/Tc in `temps` (T/Tc = 0.7 with the
    g rates sigma_eps = 1.4, sigma_p = 1.8, inside the model's stable range),
    FP64 and FP32 storage. Per droplet (periodic connected components of
    rho > (rho_v + rho_l) / 2): the interior state at its densest node, the
    equimolar radius R = sqrt(A / pi) with A the sum of (rho - rho_vb) /
    (rho_in - rho_vb) over the droplet grown by 4 nodes, and the pressure jump
    p(rho_in, T_in) - p(rho_vb, T_vb) from Eq. 17 (library host code), rho_vb,
    T_vb the medians over vapour nodes at least 12 nodes from any liquid. The
    slope of dp against 1/R is compared with the square-gradient surface
    tension at the vapour's temperature; spurious currents are max |u| / c."""
    import torch
    from scipy import ndimage
    from paper_2106_01557_gb300 import inputs, lbm
    rows = []
    for tr in temps:
        rates = SWEEP_RATES if tr < 0.75 else {}
        res = {"Tr": tr, "rates": rates}
        fields = {}
        for prec in precisions:
            cfg = lbm.default_config(n, n, precision=prec, Tr0=tr, **rates)
            lat = lbm.Lattice(cfg)
            p = lat.params()
            centers, radii = inputs.place_droplets(n, n, ndrop, 20.0, 80.0, 8.0, seed)
            rho = inputs.droplets(n, n, p["rho_v"], p["rho_l"], centers, radii, 4.0)
            z = np.zeros_like(rho)
            lat.set_fields(rho, z, z, z + p["T0"])
            t0 = time.perf_counter()
            lat.step(steps)
            lat.synchronize()
            wall = time.perf_counter() - t0
            m = lat.moments()
            lat.close()
            r, T = m["rho"], m["T"]
            fields[prec] = r
            mid = 0.5 * (p["rho_v"] + p["rho_l"])
            lab, ids = _periodic_labels(r > mid)
            vap = ndimage.distance_transform_edt(r <= mid) >= 12.0
            rvb, Tvb = float(np.median(r[vap])), float(np.median(T[vap]))
            pv = lbm.eos_pressure(cfg, rvb, Tvb)
            drops = []
            for k in ids:
                own = lab == k
                iy, ix = np.unravel_index(np.argmax(np.where(own, r, -1.0)), r.shape)
                rin, Tin = float(r[iy, ix]), float(T[iy, ix])
                grown = ndimage.binary_dilation(own, iterations=4)
                area = float(((r[grown] - rvb) / (rin - rvb)).sum())
                R = math.sqrt(max(area, 1e-12) / math.pi)
                drops.append({"R": R, "rho_in": rin, "T_in": Tin, "dp": lbm.eos_pressure(cfg, rin, Tin) - pv})
            inv_r = np.array([1.0 / d["R"] for d in drops])
            dp = np.array([d["dp"] for d in drops])
            sigma = lbm.surface_tension(cfg, Tvb / p["Tc"])
            slope, icpt = (np.polyfit(inv_r, dp, 1) if len(drops) >= 2 else (float("nan"), float("nan")))
            umax = float(np.hypot(m["ux"], m["uy"]).max() / p["c"])
            res[prec] = {"droplets_left": len(drops), "R_range": [min(d["R"] for d in drops), max(d["R"] for d in drops)],
                         "slope_over_sigma_minus_1": float(slope / sigma - 1), "sigma_theory": sigma,
                         "intercept_over_dp_min": float(icpt / dp.min()), "max_u_over_c": umax,
                         "Tr_vapour": Tvb / p["Tc"], "wall_s": wall,
                         "per_droplet": [{k: round(v, 6) for k, v in d.items()} for d in drops]}
        if "f64" in fields and "f32" in fields:
            res["f32_vs_f64_max_rho_err"] = float(np.abs(fields["f32"] - fields["f64"]).max() / fields["f64"].max())
        rows.append(res)
    return {"metric": "Laplace law, static droplets in one periodic box", "n": n, "droplets": ndrop,
            "steps": steps, "seed": seed, "results": rows}


def stefan_study(times=None, nx=8, ny=1024, precision="f64"):
    """The one-dimensional Stefan problem of Eq. 20, 21 at the paper's size
    (1024 nodes along the heating, 8 across), run to the four times of its
    Fig. 1: the open bottom at T_r 0.85 (outflow at the liquid's saturation
    pressure) below vapour, liquid at T_r 0.8, c_v = 11.2 R so that Ste =
    0.005 with the model's latent heat. The front X (where rho crosses the
    mean of the coexistence densities, from the boundary at y = -1/2)
    against X = 2 k sqrt(alpha_v (t + t0)), k the root of Eq. 21 and t0 set
    by the initial front at X0 = 20.5."""
    from paper_2106_01557_gb300 import lbm
    Tr1, Ste, cv = 0.85, 0.005, 11.2
    times = times or [4.01e6, 8.03e6, 12.04e6, 16.06e6]
    cfg = lbm.default_config(nx, ny, precision=precision, walls=1, open_sides=1, Tr_open=Tr1, c_v=cv)
    lat = lbm.Lattice(cfg)
    p = lat.params()
    T0, T1 = p["T0"], Tr1 * p["Tc"]
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    X0 = 20.0
    rho = p["rho_v"] + (p["rho_l"] - p["rho_v"]) * 0.5 * (1 + np.tanh(2 * (y - X0) / 10.0))
    T = np.where(y < X0, T1 + (T0 - T1) * (y + 0.5) / (X0 + 0.5), T0)
    lat.set_fields(rho, 0 * rho, 0 * rho, T)
    # the Stefan number with the model's latent heat a (rho_l - rho_v) + p_s (1/rho_v - 1/rho_l)
    h_lv = p["a"] * (p["rho_l"] - p["rho_v"]) + p["p_s"] * (1 / p["rho_v"] - 1 / p["rho_l"])
    ste = p["rho_v"] * p["cv"] * (T1 - T0) / (p["rho_l"] * h_lv)
    f = lambda k: k * math.sqrt(math.pi) * math.exp(k * k) * math.erf(k) - Ste
    lo, hi = 1e-12, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) < 0 else (lo, mid)
    k = 0.5 * (lo + hi)
    alpha_v = (4 + 3 * cfg.gamma1 + 2 * cfg.gamma2) / 6 * p["Cref"] * p["c"] * cfg.tau_j_v / (p["rho_v"] * p["cv"])
    t0 = (X0 + 0.5) ** 2 / (4 * k * k * alpha_v)
    mid_rho = 0.5 * (p["rho_v"] + p["rho_l"])
    rows, done, t_start = [], 0, time.perf_counter()
    for t in times:
        n = int(round(t / p["dt"]))
        lat.step(n - done)
        done = n
        r = lat.moments()["rho"].mean(axis=1)
        j = int(np.argmax(r > mid_rho))
        X = j - 0.5 + (mid_rho - r[j - 1]) / (r[j] - r[j - 1])
        Xa = 2 * k * math.sqrt(alpha_v * (t + t0))
        rows.append({"t": t, "steps": n, "X": X, "X_eq20": Xa, "rel_err": X / Xa - 1})
    lat.close()
    return {"metric": "Stefan front (Eq. 20) on the GPU path", "lattice": [nx, ny], "storage": precision,
            "Ste": ste, "k": k, "alpha_v": alpha_v, "t0": t0, "wall_s": time.perf_counter() - t_start,
            "fronts": rows}


def precision_study(checkpoints=(1000, 10000, 100000)):
    """The storage formats on the boiling workload over long runs: FP64,
    FP32, FP16S and BF16S lattices (the 16-bit ones with stochastic
    rounding, the default, and rounded to nearest: "_rn") stepped side by
    side to each checkpoint.
    Per format and checkpoint: the field errors against FP64 (max and rms of
    |x - x64| over the field's scale; for u over c) and observables that a
    moving interface does not scramble: the vapour fraction (nodes below the
    mean of the Maxwell densities), the relative drift of mass and of total
    energy from the conservation record, and the mean temperature. A format
    whose step record flags a node (non-positive or non-finite density or
    temperature) is reported with the number of such nodes and the first
    checkpoint at which it happened, and followed on."""
    import torch
    from paper_2106_01557_gb300 import lbm
    precs = ("f64", "f32", "f16s", "f16s_rn", "bf16s", "bf16s_rn")
    lats, c0 = {}, {}
    stream = torch.cuda.Stream()
    for prec in precs:
        lat, fields = boiling_case(lbm, NX, NY, prec.split("_")[0], stream_ptr=stream.cuda_stream,
                                   rounding=0 if prec.endswith("_rn") else 1)
        lat.set_fields(*fields)
        lats[prec] = lat
        c0[prec] = lat.conservation()
    p = lats["f64"].params()
    mid, c = 0.5 * (p["rho_v"] + p["rho_l"]), p["c"]
    out, done, t0 = [], 0, time.perf_counter()
    flagged = {}

    def moments(prec, cp):
        try:
            return lats[prec].moments()
        except lbm.LbmError as e:
            if e.code != -4:
                raise
            # the step record counted bad nodes; the fields are still readable
            flagged.setdefault(prec, {"first_checkpoint": cp, "bad_nodes": int(lats[prec].step_stats()[6])})
            return lats[prec].moments()
    for cp in checkpoints:
        for prec in precs:
            lats[prec].step(cp - done)
        done = cp
        ms = {prec: moments(prec, cp) for prec in precs}
        print(f"precision study: {cp} steps, flagged {flagged}", file=sys.stderr, flush=True)
        ref = ms["f64"]
        row = {"steps": cp}
        for prec in precs:
            m, cr = ms[prec], lats[prec].conservation(allow_diverged=prec in flagged)
            rec = {"vapour_fraction": float((m["rho"] < mid).mean()),
                   "mass_drift": float(cr[0] / c0[prec][0] - 1),
                   "energy_drift": float(cr[4] / c0[prec][4] - 1),
                   "mean_T_over_Tc": float(m["T"].mean() / p["Tc"])}
            if prec in flagged:
                rec["flagged"] = flagged[prec]
            if prec != "f64":
                for f in ("rho", "T"):
                    d = m[f] - ref[f]
                    scale = np.abs(ref[f]).max()
                    rec[f"err_{f}_max"] = float(np.abs(d).max() / scale)
                    rec[f"err_{f}_rms"] = float(np.sqrt((d * d).mean()) / scale)
                du = np.hypot(m["ux"] - ref["ux"], m["uy"] - ref["uy"])
                rec["err_u_over_c_max"] = float(du.max() / c)
                rec["err_u_over_c_rms"] = float(np.sqrt((du * du).mean()) / c)
            row[prec] = rec
        out.append(row)
    for lat in lats.values():
        lat.close()
    return {"metric": "storage formats against FP64 over long runs", "workload": f"boiling {NX}x{NY}",
            "wall_s": time.perf_counter() - t0, "checkpoints": out}


def cpu_baseline(seconds=12.0):
    """The FP64 oracle as it stands, on this host's cores, on a bounded
    slice of the workload (4096 x 64 rows of the same layout with walls)."""
    from oracle import Oracle, thermo
    from paper_2106_01557_gb300 import inputs
    nx, ny = 4096, 64
    cfg = thermo.Config(nx=nx, ny=ny, walls=1, accel_y=-1e-5, Tr_bottom=0.8, Tr_hot=0.95,
                        hot_x0=inputs.hot_spot_x0(nx, 32, seed=3), hot_len=32)
    o = Oracle(cfg)
    p = o.p
    rho = inputs.layer(nx, ny, p.rho_v, p.rho_l, 48.0, 4.0)
    o.init_fields(rho, 0 * rho, 0 * rho, 0 * rho + p.T0)
    o.step(1)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        o.step(2)
        steps += 2
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": nx * ny * steps / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{nx}x{ny} slice of the workload, {steps} steps, FP64, OpenMP over rows"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f64", "f32", "f16s", "bf16s"])
    ap.add_argument("--rounding", type=int, default=1, choices=[0, 1],
                    help="16-bit storage: 1 stochastic rounding (the library default), 0 nearest")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--variant-steps", type=int, default=1000,
                    help="steps of each storage format for the error-vs-FP64 comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-study", type=int, default=0,
                    help="run the 256-case sweep for this many steps and report coexistence per case")
    ap.add_argument("--batch-precision", default="f16s", choices=["f32", "f16s", "bf16s"])
    ap.add_argument("--precision-study", type=int, default=0,
                    help="run FP64/FP32/FP16S/BF16S side by side to 1,000, 10,000 and this many steps; print the errors")
    ap.add_argument("--droplet-study", type=int, default=0,
                    help="box size n: a droplet of diameter n/4 evaporating in an n x n box heated on all sides")
    ap.add_argument("--laplace-study", type=int, default=0,
                    help="run eight static droplets in a periodic 512 x 512 box for this many steps (T/Tc 0.7, 0.8, 0.9; FP64 and FP32)")
    ap.add_argument("--droplet-pair-study", type=int, default=0,
                    help="box size n: the paper's large-small droplet pair scaled by n/1024, Ste 0.005, 0.05, 0.5")
    ap.add_argument("--stefan-study", action="store_true",
                    help="run the 1-D Stefan problem to the paper's Fig. 1 times and report the front against Eq. 20")
    ap.add_argument("--stefan-precision", default="f64", choices=["f64", "f32"])
    ap.add_argument("--surrogate-ks", default="100,200",
                    help="jump lengths K of the extra surrogate studies (comma list; empty: none)")
    ap.add_argument("--surrogate-iters", type=int, default=3000,
                    help="training iterations of the surrogate study in the default run (0: skip)")
    ap.add_argument("--nx", type=int, default=NX, help="smaller lattice for profiling captures")
    ap.add_argument("--ny", type=int, default=NY)
    args = ap.parse_args()
    set_size(args.nx, args.ny)
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.batch_study:
        if rank == 0:
            print(json.dumps(batch_study(args.batch_study, precision=args.batch_precision)))
        return
    if args.droplet_pair_study:
        if rank == 0:
            res = droplet_pair_study(n=args.droplet_pair_study,
                                     report=lambda case: print(json.dumps({"case": case}), flush=True))
            print(json.dumps({k: v for k, v in res.items() if k != "results"}))
        return
    if args.laplace_study:
        if rank == 0:
            print(json.dumps(laplace_study(steps=args.laplace_study)))
        return
    if args.stefan_study:
        if rank == 0:
            print(json.dumps(stefan_study(precision=args.stefan_precision)))
        return
    if args.droplet_study:
        if rank == 0:
            n = args.droplet_study
            print(json.dumps(droplet_study(n=n, D0=n / 4)))
        return
    if args.precision_study:
        if rank == 0:
            cps = tuple(sorted({k for k in (1000, 10000, args.precision_study) if k <= args.precision_study}))
            print(json.dumps(precision_study(cps)))
        return
    config = {"workload": f"boiling {NX}x{NY}, walls, hot spot 32 cells, g=1e-5, {args.precision.upper()} storage",
              "nx": NX, "ny": NY, "precision": args.precision,
              "l2": "state (2 x 302 MB FP32) larger than L2; no flush needed",
              "parallelism": f"replicas x{world}"}

    if args.impl == "reference":
        if rank != 0:
            return
        import torch  # noqa: F401  (only to keep the launch identical)
        per = []
        for _ in range(args.warmup):
            pass
        for _ in range(max(1, args.steps if args.steps <= 3 else 3)):
            per.append(cpu_baseline(seconds=8.0))
        v = float(np.median([p["value"] for p in per]))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS",
                "n_gpus": args.gpus, "steps": len(per), "warmup": args.warmup, "higher_is_better": True,
                "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": {"kind": "oracle", "cores": per[0]["cores"], "sample": per[0]["sample"], "value": v},
                "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank != 0:
        return
    peaks, kind = measured_peaks()
    hbm = hbm_peak(peaks)
    achieved = res["bytes_step"] / (res["ms_step"] * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": res["mlups"], "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f32": "f32", "f16s": "f16 storage / f32 math",
                  "bf16s": "bf16 storage / f32 math"}[args.precision],
        "data": "synthetic", "config": config,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": step_traffic(), "traffic_unit": "DRAM bytes per launch (ncu capture)", "peak_kind": kind,
                     "algorithmic_bytes_per_lu": res["bytes_step"] / (NX * NY),
                     "timing": "CUDA events over the timed steps on the launching stream / steps"},
        "gpu_launches": args.steps,
        "clocks": res["clocks"], "e2e": res["e2e"],
        "variants": sorted(res["variants"]),
        "conservation_last_step": res["stats"],
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    # the variants and studies first, one JSON line each; the headline last
    for name, v in res["variants"].items():
        print(json.dumps({"variant": name, "result": v}))
    print(json.dumps(line))


if __name__ == "__main__":
    main()
