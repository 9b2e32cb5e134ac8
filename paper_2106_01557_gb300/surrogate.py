"""Training data, training loop and rollout study of the learned surrogate.

Data: periodic 256 x 256 boxes with 1-4 liquid droplets (radius 15-50, at
T/Tc = 0.8 and the Maxwell liquid density) in vapour superheated to an
ambient T/Tc in [0.85, 0.95]; the droplets evaporate. All runs advance
together as one batch (lbm_batch_*, FP32); snapshots of (rho, u, T) every K
steps give the (input, target) pairs. The LB constants of every run are
those of T_r0 = 0.8.

Every array operation on the fields here is data movement (stacking,
casting, indexing); the model's arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs, lbm


def droplet_case(nx, ny, p, seed, n_drop=None, r_lo=15.0, r_hi=50.0, tr_amb=None, rng=None):
    """(rho, u_x, u_y, T) of an evaporation case: droplets at T0 in vapour at
    an ambient reduced temperature (seeded)."""
    rng = rng or np.random.default_rng(seed)
    n_drop = n_drop or int(rng.integers(1, 5))
    tr_amb = tr_amb if tr_amb is not None else float(rng.uniform(0.85, 0.95))
    centers, radii = inputs.place_droplets(nx, ny, n_drop, r_lo, r_hi, 12.0, seed)
    rho = inputs.droplets(nx, ny, p["rho_v"], p["rho_l"], centers, radii, 4.0)
    liquid = (rho - p["rho_v"]) / (p["rho_l"] - p["rho_v"])
    T = p["T0"] + (tr_amb * p["Tc"] - p["T0"]) * (1.0 - liquid)
    z = np.zeros_like(rho)
    return rho, z, z.copy(), T


def norm_consts(p):
    """Offsets and scales of (rho, u_x, u_y, T) for the network."""
    return ([p["rho_v"], 0.0, 0.0, p["T0"]],
            [p["rho_l"] - p["rho_v"], 0.01 * p["c"], 0.01 * p["c"], 0.1 * p["Tc"]])


def generate_pairs(n_runs=40, pairs_per_run=50, K=50, size=256, seed=10, warmup=200):
    """Returns a float32 CUDA tensor of snapshots (runs, pairs + 1, 4, size,
    size) and the case parameters; pair j of run r is (snap[r, j], snap[r, j+1]).
    The first `warmup` steps (the relaxation of the initial tanh interfaces)
    are not sampled."""
    import torch
    cfg = lbm.default_config(size, size, precision="f32")
    probe = lbm.Lattice(cfg)
    p = probe.params()
    probe.close()
    b = lbm.Batch([cfg] * n_runs)
    for r in range(n_runs):
        b.set_fields(r, *droplet_case(size, size, p, seed + r))
    if warmup:
        b.step(warmup)
    snaps = torch.empty((n_runs, pairs_per_run + 1, 4, size, size), dtype=torch.float32, device="cuda")
    for j in range(pairs_per_run + 1):
        if j:
            b.step(K)
        for r in range(n_runs):
            m = b.moments(r)
            snaps[r, j] = torch.from_numpy(np.stack([m["rho"], m["ux"], m["uy"], m["T"]]).astype(np.float32))
    b.close()
    return snaps, p


def train(sur, snaps, iters=1000, batch=8, lr=1e-3, seed=0, log_every=100, holdout_runs=4):
    """Adam on random minibatches of pairs from all but the last holdout_runs
    runs; returns (losses, holdout loss)."""
    import torch
    rng = np.random.default_rng(seed)
    R, J = snaps.shape[0] - holdout_runs, snaps.shape[1] - 1
    losses = []
    t0 = time.perf_counter()
    for it in range(iters):
        # linear warm-up over the first 5% of the iterations, then cosine decay
        warm = max(1, iters // 20)
        lr_it = lr * min(1.0, (it + 1) / warm) * 0.5 * (1.0 + math.cos(math.pi * it / iters))
        r = rng.integers(0, R, size=batch)
        j = rng.integers(0, J, size=batch)
        x = snaps[r, j].permute(1, 0, 2, 3).contiguous().double()
        y = snaps[r, j + 1].permute(1, 0, 2, 3).contiguous().double()
        losses.append(sur.train_step(x, y, lr_it))
        if log_every and it % log_every == 0:
            pass
    train_s = time.perf_counter() - t0
    hold = []
    for r in range(R, snaps.shape[0]):
        x = snaps[r, :J].permute(1, 0, 2, 3).contiguous().double()
        y = snaps[r, 1:].permute(1, 0, 2, 3).contiguous().double()
        for k in range(0, J, 8):
            hold.append(sur.loss_grad(x[:, k:k + 8].contiguous(), y[:, k:k + 8].contiguous(), grads=False)[0])
    return np.array(losses), float(np.mean(hold)) if hold else None, train_s


def persistence_loss(sur, snaps, holdout_runs=4):
    """Loss of the trivial predictor 'no change' on the holdout pairs, in the
    network's normalisation: the bar a trained network must beat."""
    off, scale = sur.norm_off, sur.norm_scale
    J = snaps.shape[1] - 1
    out = []
    for r in range(snaps.shape[0] - holdout_runs, snaps.shape[0]):
        d = (snaps[r, 1:] - snaps[r, :J]).double().cpu().numpy()
        for c in range(4):
            d[:, c] /= scale[c]
        out.append(np.mean(d ** 2))
    return float(np.mean(out))


def interface_stats(m, p):
    """Liquid mask (nodes with rho above the mid density) and the number of
    liquid-vapour edges between x- and y-neighbours (periodic)."""
    liq = m["rho"] > 0.5 * (p["rho_v"] + p["rho_l"])
    edges = int((liq != np.roll(liq, -1, axis=0)).sum() + (liq != np.roll(liq, -1, axis=1)).sum())
    return liq, edges


def network_cost(P, C=64, B=6):
    """Algorithmic work of one forward pass over P pixels: the FLOPs of its
    3x3 convolutions at their real channel counts (lift 4 -> C, 2 B
    convolutions C -> C, projection C -> 4), and the HBM bytes if every
    layer reads its inputs once and writes its output once: FP64 fields in
    and out, the packed input (16 BF16 channels and its FP32 copy), each
    BF16 activation written once and read by the next layer (the second
    convolution of a block also reads the block's input as residual), and
    the 16-channel FP32 output."""
    flops = 2 * 9 * P * (4 * C + 2 * B * C * C + C * 4)
    act = P * C * 2
    nbytes = (4 * 8 * P + P * 16 * 2 + P * 4 * 4)   # pack
    nbytes += P * 16 * 2 + act                          # lift
    nbytes += B * (2 * act) + B * (3 * act)             # blocks
    nbytes += act + P * 4 * 4 + P * 16 * 4              # projection with the FP32 residual
    nbytes += P * 16 * 4 + 4 * 8 * P                    # unpack
    return flops, nbytes


def lb_own_drift(cfg, fields, p, njumps, K):
    """What the plain LB does per K-step jump on the same case: the largest
    relative change of mass and total energy, and the largest mean interface
    displacement (nodes that changed phase) / ((pi/4) edges), in lattice units."""
    lat = lbm.Lattice(cfg)
    lat.set_fields(*fields)
    lat.step(2)
    c0 = lat.conservation()
    a0, e0 = interface_stats(lat.moments(), p)
    dm = de = da = 0.0
    for _ in range(njumps):
        lat.step(K)
        c1 = lat.conservation()
        a1, e1 = interface_stats(lat.moments(), p)
        dm = max(dm, abs(c1[0] / c0[0] - 1.0))
        de = max(de, abs(c1[4] / c0[4] - 1.0))
        da = max(da, int((a1 != a0).sum()) / (0.25 * math.pi * max(e0, 1)))
        c0, a0, e0 = c1, a1, e1
    lat.close()
    return {"mass": dm, "energy": de, "iface_displacement": da}


def identity_local_change(sur, cfg, fields, K, kv, njumps=2):
    """The local change the verification steps make to an LB state that was
    only read out and re-initialised (a network that predicts no change):
    the floor under the rollout's local check."""
    ident = lbm.Surrogate(sur.norm_off, sur.norm_scale, K=K, blocks=sur.blocks, conserve_mass=sur.conserve_mass)
    prm = sur.get_params().copy()
    nproj = 9 * 4 * sur.channels + 4
    prm[-nproj:] = 0.0                        # zero projection: y = x
    ident.set_params(prm)
    lat = lbm.Lattice(cfg)
    lat.set_fields(*fields)
    st = ident.rollout(lat, njumps, 1.0, 1e3, verify_steps=kv, field_tol=1e3)
    lat.close()
    ident.close()
    return {"rho": st["max_local_change_rho_all"], "T": st["max_local_change_T_all"]}


def rollout_study(sur, p, size=1024, njumps=10, K=50, tol=1e-3, iface_tol=0.5, seed=99, n_drop=24,
                  field_tol=0.2):
    """Surrogate rollout with LB fallback against the plain LB over the same
    njumps * (K + K/10) steps (each jump: K steps predicted, K/10 LB
    verification steps) on a size x size evaporation case: wall time of
    both, fallbacks, the field error of the surrogate path against the LB,
    and the LB's own per-jump drift and local change beside the thresholds."""
    import torch
    kv = max(1, K // 10)
    cfg = lbm.default_config(size, size, precision="f32")
    fields = droplet_case(size, size, p, seed, n_drop=n_drop)
    own = lb_own_drift(cfg, fields, p, njumps, K + kv)
    own_local = identity_local_change(sur, cfg, fields, K, kv)
    ref = lbm.Lattice(cfg)
    ref.set_fields(*fields)
    ref.step(2)
    ref.synchronize()
    t0 = time.perf_counter()
    ref.step(njumps * (K + kv))
    ref.synchronize()
    t_lb = time.perf_counter() - t0
    m_ref = ref.moments()
    ref.close()
    lat = lbm.Lattice(cfg)
    lat.set_fields(*fields)
    lat.step(2)
    lat.synchronize()
    t0 = time.perf_counter()
    try:
        st = sur.rollout(lat, njumps, tol, iface_tol, verify_steps=kv, field_tol=field_tol)
    except lbm.LbmError as e:  # the fallback LB steps diverged from an accepted surrogate state
        lat.close()
        return {"size": size, "jumps": njumps, "K": K, "verify_steps": kv, "error": str(e),
                "lb_own_max_drift_per_jump": own}
    t_sur = time.perf_counter() - t0
    m = lat.moments()
    lat.close()
    # forward pass alone (the network's share of a jump)
    x = torch.from_numpy(np.stack([m["rho"], m["ux"], m["uy"], m["T"]])[:, None]).cuda().contiguous()
    out = torch.empty_like(x)
    sur.forward(x, out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        sur.forward(x, out)
    torch.cuda.synchronize()
    t_fwd = (time.perf_counter() - t0) / 5
    # the same network on the warp-level mma.sync convolutions
    alt = lbm.Surrogate(sur.norm_off, sur.norm_scale, K=K, conv_path="mma", conserve_mass=sur.conserve_mass)
    alt.set_params(sur.get_params())
    alt.forward(x, out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        alt.forward(x, out)
    torch.cuda.synchronize()
    t_fwd_mma = (time.perf_counter() - t0) / 5
    alt.close()
    flops, nbytes = network_cost(size * size)
    c = p["c"]
    err = {"rho": float(np.abs(m["rho"] - m_ref["rho"]).max() / np.abs(m_ref["rho"]).max()),
           "T": float(np.abs(m["T"] - m_ref["T"]).max() / np.abs(m_ref["T"]).max()),
           "u_over_c": float(max(np.abs(m["ux"] - m_ref["ux"]).max(), np.abs(m["uy"] - m_ref["uy"]).max()) / c),
           "rho_rms": float(np.sqrt(np.mean((m["rho"] - m_ref["rho"]) ** 2)) / np.abs(m_ref["rho"]).max())}
    return {"size": size, "jumps": njumps, "K": K, "verify_steps": kv, "drift_tol": tol, "iface_tol": iface_tol,
            "lb_s": t_lb, "surrogate_path_s": t_sur, "speedup_vs_lb": t_lb / t_sur,
            "accepted": st["accepted"], "fallbacks": st["fallbacks"],
            "ms_in_rollout": {"read_state": st["ms_read_state"], "network": st["ms_network"],
                              "check_and_reinit": st["ms_check_reinit"], "verify_steps": st["ms_verify"],
                              "fallback_lb": st["ms_fallback_lb"]},
            "ms_per_jump_network_only": 1e3 * t_fwd, "ms_per_jump_network_mma_sync": 1e3 * t_fwd_mma,
            "network_forward": {"flops": flops, "bytes": nbytes, "tflops": flops / t_fwd / 1e12,
                                "gbs": nbytes / t_fwd / 1e9},
            "ms_per_jump_lb_steps": 1e3 * t_lb / njumps,
            "max_mass_drift_accepted": st["max_mass_drift"], "max_energy_drift_accepted": st["max_energy_drift"],
            "max_drift_all_jumps": {"mass": st["max_mass_drift_all"], "energy": st["max_energy_drift_all"],
                                    "iface_displacement": st["max_iface_displacement_all"]},
            "max_local_change_all_jumps": {"rho": st["max_local_change_rho_all"],
                                           "T": st["max_local_change_T_all"], "field_tol": field_tol},
            "lb_own_max_drift_per_jump": own, "lb_own_local_change_after_reinit": own_local,
            "unphysical": st["unphysical"], "err_vs_lb": err}


def init_params(channels=64, blocks=6, seed=0):
    """Seeded He-normal initial weights in the library's parameter order; the
    projection starts small so the untrained network is near the identity."""
    rng = np.random.default_rng(seed)
    parts = []

    def conv(ci, co, s=1.0):
        parts.append(rng.normal(0.0, s * math.sqrt(2.0 / (9 * ci)), size=9 * co * ci))
        parts.append(np.zeros(co))

    conv(4, channels)
    for _ in range(blocks):
        conv(channels, channels)
        conv(channels, channels, 0.1)
    conv(channels, 4, 0.1)
    return np.concatenate(parts).astype(np.float32)


def study(iters=1000, n_runs=40, pairs_per_run=50, K=50, size=256, rollout_size=1024, njumps=10, tol=1e-3,
          seed=0, lr=1e-3, batch=8):
    """Generate data, train from seeded initial weights, evaluate on held-out
    runs against persistence, and run the rollout study."""
    t0 = time.perf_counter()
    snaps, p = generate_pairs(n_runs, pairs_per_run, K, size, seed=seed + 10)
    t_data = time.perf_counter() - t0
    off, scale = norm_consts(p)
    sur = lbm.Surrogate(off, scale, K=K)
    sur.set_params(init_params(seed=seed))
    losses, hold, t_train = train(sur, snaps, iters=iters, batch=batch, lr=lr, seed=seed)
    pers = persistence_loss(sur, snaps)
    roll = rollout_study(sur, p, size=rollout_size, njumps=njumps, K=K, tol=tol)
    out = {"params": sur.num_params, "pairs": n_runs * pairs_per_run, "data_s": t_data,
           "train_iters": iters, "batch": batch, "train_s": t_train, "ms_per_train_iter": 1e3 * t_train / iters,
           "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-20:])),
           "holdout_loss": hold, "persistence_loss": pers,
           "holdout_gain_vs_persistence": pers / hold if hold else None, "rollout": roll}
    sur.close()
    return out
