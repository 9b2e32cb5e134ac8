"""The learned surrogate's BF16 tensor-core kernels against its FP64 oracle
network: forward pass, loss and every parameter gradient, on both
convolution paths (tcgen05 with tensor-memory accumulators, warp-level
mma.sync); sampled windows of a full-size 1024 x 1024 forward pass; then
training and the rollout with LB fallback."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


PATHS = ["tcgen05", "mma"]


def _make(channels=64, blocks=2, seed=0, K=10, conv_path="tcgen05", conserve_mass=False):
    from oracle import surrogate as S
    from paper_2106_01557_gb300 import lbm
    p = S.init_params(channels=channels, blocks=blocks, seed=seed)
    # a projection large enough that the network output differs from its input
    rng = np.random.default_rng(seed + 100)
    p["proj"] = (rng.normal(0, 0.05, p["proj"][0].shape), rng.normal(0, 0.05, p["proj"][1].shape))
    s = lbm.Surrogate([0, 0, 0, 0], [1, 1, 1, 1], K=K, channels=channels, blocks=blocks, conv_path=conv_path,
                      conserve_mass=conserve_mass)
    s.set_params(lbm.surrogate_params_from_oracle_layout(p))
    return S, p, s


def _fields(N, H, W, seed):
    rng = np.random.default_rng(seed)
    # smooth-ish normalised fields
    x = rng.normal(size=(N, H, W, 4))
    x = 0.5 * (x + np.roll(x, 1, axis=2))
    return x


def _to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.moveaxis(x, -1, 0))).cuda()


# BF16 operands and activations with FP32 accumulation: the network's
# change of the fields, element by element, within 2% of its largest value,
# and every gradient tensor, element by element, within 5% of its largest
# entry (measured: forward up to 0.6%, gradients up to 3.0%)
FWD_TOL, GRAD_TOL = 2e-2, 5e-2


def _close(d, d_ref):
    assert np.abs(d - d_ref).max() < FWD_TOL * np.abs(d_ref).max(), np.abs(d - d_ref).max() / np.abs(d_ref).max()


# (N, H, W): one partial 128-pixel strip; several strips with a ragged 16-pixel
# tail and more rows than CTAs, so runs of rows cross strip and image borders
SHAPES = [(2, 8, 32), (3, 20, 272)]


@pytest.mark.parametrize("conserve_mass", [False, True])
@pytest.mark.parametrize("conv_path", PATHS)
@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_oracle(gpu_lib, conv_path, shape, conserve_mass):
    import torch
    S, p, s = _make(conv_path=conv_path, conserve_mass=conserve_mass)
    x = _fields(*shape, 1)
    y_ref, _ = S.forward(p, x, conserve_mass)
    out = torch.empty((4,) + shape, dtype=torch.float64, device="cuda")
    s.forward(_to_dev(x), out)
    y = np.moveaxis(out.cpu().numpy(), 0, -1)
    _close(y - x, y_ref - x)


@pytest.mark.parametrize("shape", SHAPES + [(1, 300, 1024)])
def test_conv_paths_bit_identical(gpu_lib, shape):
    # both convolution paths sum each output's 9 CIN / 16 K-steps in the same
    # (dy, dx, channel chunk) order, each step a K = 16 product of BF16
    # operands with FP32 accumulation: the forward output agrees bit for bit,
    # and so do the gradients (the weight and bias gradients sum their
    # per-block partials in a fixed order). The 1 x 300 x 1024
    # case gives each CTA a run of about 16 rows of eight 128-pixel strips,
    # some runs going on from one strip into the next.
    import torch
    x = _to_dev(_fields(*shape, 11))
    t = _to_dev(_fields(*shape, 12))
    outs, grads = [], []
    for path in PATHS:
        S, p, s = _make(seed=13, conv_path=path)
        out = torch.empty((4,) + shape, dtype=torch.float64, device="cuda")
        s.forward(x, out)
        outs.append(out)
        grads.append(s.loss_grad(x, t)[1])
    assert torch.equal(outs[0], outs[1])
    assert np.array_equal(grads[0], grads[1])


def test_forward_full_size_sampled_windows(gpu_lib):
    # 1024 x 1024 (the rollout size): every CTA walks long runs of rows.
    # The output at a pixel depends only on inputs within R = 2 B + 2 pixels
    # (B blocks of two 3 x 3 convolutions, plus lift and projection), so the
    # oracle on a crop of the periodic input, R pixels wider on each side,
    # gives the exact output on the crop's centre.
    import torch
    S, p, s = _make(blocks=2, seed=5)
    R, h = 2 * 2 + 2, 32
    x = _fields(1, 1024, 1024, 6)
    out = torch.empty((4, 1, 1024, 1024), dtype=torch.float64, device="cuda")
    s.forward(_to_dev(x), out)
    y = np.moveaxis(out.cpu().numpy(), 0, -1)
    for (yc, xc) in [(0, 0), (500, 640), (1000, 1016)]:
        crop = np.roll(x, (R - yc, R - xc), axis=(1, 2))[:, :h + 2 * R, :h + 2 * R]
        y_ref, _ = S.forward(p, crop)
        got = np.roll(y, (-yc, -xc), axis=(1, 2))[:, :h, :h]
        ref = y_ref[:, R:R + h, R:R + h]
        _close(got - crop[:, R:R + h, R:R + h], ref - crop[:, R:R + h, R:R + h])


def test_mass_layer_keeps_each_images_mass(gpu_lib):
    # the density sums of input and output agree per image to FP32 rounding
    # of the normalised fields; without the layer the network moves them
    import torch
    x = _fields(3, 20, 272, 8)
    sums = {}
    for cm in (False, True):
        S, p, s = _make(seed=9, conserve_mass=cm)
        out = torch.empty((4, 3, 20, 272), dtype=torch.float64, device="cuda")
        s.forward(_to_dev(x), out)
        sums[cm] = out[0].sum(dim=(1, 2)).cpu().numpy()
    ref = x[..., 0].sum(axis=(1, 2))
    scale = np.abs(x[..., 0]).sum(axis=(1, 2))
    assert np.abs(sums[True] - ref).max() < 1e-6 * scale.max()
    assert np.abs(sums[False] - ref).min() > 1e-3 * scale.min()


@pytest.mark.parametrize("conserve_mass", [False, True])
@pytest.mark.parametrize("conv_path", PATHS)
@pytest.mark.parametrize("shape", SHAPES)
def test_gradients_match_oracle(gpu_lib, conv_path, conserve_mass, shape):
    # every weight and bias gradient; the second shape has several 128-pixel
    # strips with a ragged 16-pixel tail and more row chunks than CTAs
    S, p, s = _make(seed=3, conv_path=conv_path, conserve_mass=conserve_mass)
    x = _fields(*shape, 4)
    t = x + 0.3 * _fields(*shape, 5)
    y_ref, cache = S.forward(p, x, conserve_mass)
    g_ref = S.flatten(S.backward(p, cache, y_ref, t))
    loss, g = s.loss_grad(_to_dev(x), _to_dev(t))
    assert loss == pytest.approx(S.loss(y_ref, t), rel=2e-2)
    off, worst = 0, 0.0
    for k, gr in enumerate(g_ref):
        n = gr.size
        gg = g[off:off + n].astype(np.float64)
        gr = gr.reshape(-1)
        off += n
        err = np.abs(gg - gr).max() / max(np.abs(gr).max(), 1e-30)
        worst = max(worst, err)
        assert err < GRAD_TOL, (k, err)
    assert off == g.size
    print(f"{conv_path} mass={conserve_mass} {shape}: largest per-tensor gradient error {worst:.3e}")


def test_training_reduces_loss(gpu_lib):
    # learn a fixed smooth map of the fields: loss falls by an order of magnitude
    import torch
    S, p, s = _make(blocks=2, seed=7)
    rng = np.random.default_rng(8)
    xs = [_fields(4, 16, 32, 20 + k) for k in range(4)]
    ts = [x + 0.2 * np.roll(x, 1, axis=1) - 0.2 * np.roll(x, -1, axis=2) for x in xs]
    dev = [(_to_dev(x), _to_dev(t)) for x, t in zip(xs, ts)]
    first = [s.loss_grad(a, b, grads=False)[0] for a, b in dev]
    for it in range(200):
        a, b = dev[it % 4]
        s.train_step(a, b, lr=2e-3)
    last = [s.loss_grad(a, b, grads=False)[0] for a, b in dev]
    assert np.mean(last) < 0.1 * np.mean(first)


def test_training_is_reproducible_bit_for_bit(gpu_lib):
    # no reduction of the training step uses atomics: two networks trained
    # from the same weights on the same minibatches give the same losses and
    # the same weights, bit for bit
    xs = [_fields(4, 16, 32, 40 + k) for k in range(3)]
    ts = [x + 0.2 * np.roll(x, 1, axis=1) for x in xs]
    dev = [(_to_dev(x), _to_dev(t)) for x, t in zip(xs, ts)]
    runs = []
    for _ in range(2):
        S, p, s = _make(blocks=2, seed=17, conserve_mass=True)
        losses = [s.train_step(*dev[it % 3], lr=1e-3) for it in range(30)]
        runs.append((losses, s.get_params()))
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])


def test_first_adam_step_is_the_textbook_update(gpu_lib):
    # from zero moments the bias-corrected Adam update (beta1 0.9, beta2
    # 0.999, eps 1e-8) is -lr g / (|g| + eps): a step of lr against the sign
    # of the gradient wherever |g| >> eps, and never longer than lr
    S, p, s = _make(blocks=2, seed=11)
    x = _fields(2, 16, 32, 30)
    t = x + 0.3 * _fields(2, 16, 32, 31)
    a, b = _to_dev(x), _to_dev(t)
    w0 = s.get_params().astype(np.float64)
    _, g = s.loss_grad(a, b)
    lr = 1e-3
    s.train_step(a, b, lr=lr)
    dw = s.get_params().astype(np.float64) - w0
    big = np.abs(g) > 1e-4
    assert big.sum() > 1000
    assert np.abs(dw[big] / lr + np.sign(g[big])).max() < 1e-2
    assert np.abs(dw).max() <= lr * (1 + 1e-3)


def test_rollout_falls_back_and_accepts(gpu_lib):
    from oracle import Oracle, thermo
    from paper_2106_01557_gb300 import inputs, lbm
    nx = ny = 64
    o = Oracle(thermo.Config(nx=nx, ny=ny))
    pp = o.p
    rho = inputs.droplets(nx, ny, pp.rho_v, pp.rho_l, [(32, 32)], [14], 4.0)
    z = np.zeros_like(rho)
    off = [pp.rho_v, 0.0, 0.0, pp.T0]
    scale = [pp.rho_l - pp.rho_v, 0.01 * pp.c, 0.01 * pp.c, 0.05 * pp.Tc]
    # an untrained network with a large projection moves the fields: rejected
    S, p, _ = _make(blocks=2, seed=11)
    p["proj"] = (p["proj"][0] * 20, p["proj"][1] * 20)
    s = lbm.Surrogate(off, scale, K=10, blocks=2)
    s.set_params(lbm.surrogate_params_from_oracle_layout(p))
    lat = lbm.Lattice.create(nx, ny, precision="f32")
    lat.set_fields(rho, z, z, np.full_like(rho, pp.T0))
    st = s.rollout(lat, 3, drift_tol=1e-3, verify_steps=2)
    assert st["fallbacks"] == 3 and st["accepted"] == 0
    assert lat.steps == 36  # every jump advances K + verify_steps
    # a network whose projection is zero is the identity: every jump is
    # accepted (the young tanh-4 droplet still relaxes fast, so the local
    # check is loosened here; it has a test of its own)
    p["proj"] = (0 * p["proj"][0], 0 * p["proj"][1])
    s.set_params(lbm.surrogate_params_from_oracle_layout(p))
    st = s.rollout(lat, 3, drift_tol=1e-3, verify_steps=2, field_tol=0.5)
    # an accepted jump counts its K predicted steps and its verification steps
    assert st["accepted"] == 3 and st["fallbacks"] == 0 and lat.steps == 36 + 3 * (10 + 2)
    assert st["max_mass_drift"] < 1e-6
    # the device's copy of the count (it keys stochastic rounding) follows
    assert lat.step_stats()[7] == lat.steps


def test_trained_network_beats_no_change_on_held_out_runs(gpu_lib):
    # the gain of the learned part over the method without it, on data the
    # network never saw: LB snapshot pairs K = 50 steps apart from evaporating
    # droplets; after a short training the network's loss on held-out runs is
    # below the loss of predicting no change (what the plain method offers in
    # the same single call)
    from paper_2106_01557_gb300 import lbm, surrogate as S
    snaps, p = S.generate_pairs(n_runs=10, pairs_per_run=20, K=50, size=256, seed=30)
    off, scale = S.norm_consts(p)
    sur = lbm.Surrogate(off, scale, K=50)
    sur.set_params(S.init_params(seed=1))
    losses, hold, _ = S.train(sur, snaps, iters=250, batch=8, lr=1e-3, seed=2, holdout_runs=2)
    pers = S.persistence_loss(sur, snaps, holdout_runs=2)
    # (the mass-conserving layer already removes the untrained network's
    # mean density error, so the loss starts lower than without it)
    assert np.mean(losses[-20:]) < 0.33 * np.mean(losses[:20])
    assert hold < pers, (hold, pers)


def test_rollout_rejects_a_moved_interface(gpu_lib):
    # a network that moves the density field one cell in +x: mass is kept
    # (a periodic shift, and the mass layer), the total energy barely changes
    # (uniform T, u = 0), so only the interface check can reject the jump;
    # a 1-cell shift of a round droplet moves its interface by 2/pi cells on
    # average, above the 0.5-cell threshold
    from oracle import Oracle, thermo
    from oracle import surrogate as S
    from paper_2106_01557_gb300 import inputs, lbm
    nx = ny = 64
    pp = Oracle(thermo.Config(nx=nx, ny=ny)).p
    rho = inputs.droplets(nx, ny, pp.rho_v, pp.rho_l, [(32, 32)], [14], 4.0)
    z = np.zeros_like(rho)
    off = [pp.rho_v, 0.0, 0.0, pp.T0]
    scale = [pp.rho_l - pp.rho_v, 0.01 * pp.c, 0.01 * pp.c, 0.05 * pp.Tc]
    p = S.init_params(channels=64, blocks=2, seed=0)
    zero = lambda a: np.zeros_like(a)
    wl = zero(p["lift"][0])
    wl[4, 0, 0] = 1.0                       # h channel 0 = normalised rho
    p["lift"] = (wl, zero(p["lift"][1]))
    p["blocks"] = [((zero(w1), zero(b1)), (zero(w2), zero(b2))) for (w1, b1), (w2, b2) in p["blocks"]]
    wp = zero(p["proj"][0])
    wp[3, 0, 0], wp[4, 0, 0] = 1.0, -1.0    # y_rho = x_rho + rho(x - 1) - rho(x)
    p["proj"] = (wp, zero(p["proj"][1]))
    s = lbm.Surrogate(off, scale, K=10, blocks=2)
    s.set_params(lbm.surrogate_params_from_oracle_layout(p))
    lat = lbm.Lattice.create(nx, ny, precision="f32")
    lat.set_fields(rho, z, z, np.full_like(rho, pp.T0))
    st = s.rollout(lat, 2, drift_tol=1e-3, iface_tol=0.5)
    assert st["fallbacks"] == 2 and st["accepted"] == 0 and st["unphysical"] == 0
    assert st["max_mass_drift_all"] < 1e-5
    assert 0.5 < st["max_iface_displacement_all"] < 0.9
    # the same jump passes a looser interface threshold
    lat.set_fields(rho, z, z, np.full_like(rho, pp.T0))
    st = s.rollout(lat, 1, drift_tol=1e-2, iface_tol=1.0)
    assert st["accepted"] == 1


def test_rollout_rejects_a_local_temperature_spike(gpu_lib):
    # A network that sharpens the temperature field, y_T = x_T + A (8 x_T -
    # sum of the 8 neighbours' x_T), turns a small warm node of a uniform
    # vapour into a one-node spike with cold neighbours. Mass is untouched,
    # the thermal energy of the spike and of its neighbours cancels and no
    # node changes phase, so the global checks pass; the LB's verification
    # steps spread the spike, and the local check rejects the jump. With the
    # local check loosened the same jump is accepted.
    from oracle import Oracle, thermo
    from oracle import surrogate as S
    from paper_2106_01557_gb300 import lbm
    nx = ny = 32
    pp = Oracle(thermo.Config(nx=nx, ny=ny)).p
    rho = np.full((ny, nx), pp.rho_v)
    z = np.zeros_like(rho)
    T = np.full_like(rho, pp.T0)
    T[16, 16] += 0.002 * pp.Tc
    off = [pp.rho_v, 0.0, 0.0, pp.T0]
    scale = [pp.rho_l - pp.rho_v, 0.01 * pp.c, 0.01 * pp.c, 0.05 * pp.Tc]
    p = S.init_params(channels=64, blocks=2, seed=0)
    zero = lambda a: np.zeros_like(a)
    wl = zero(p["lift"][0])
    wl[4, 0, 3], wl[4, 1, 3] = 1.0, -1.0        # h0 = x_T, h1 = -x_T (relu keeps each sign)
    p["lift"] = (wl, zero(p["lift"][1]))
    p["blocks"] = [((zero(w1), zero(b1)), (zero(w2), zero(b2))) for (w1, b1), (w2, b2) in p["blocks"]]
    s = lbm.Surrogate(off, scale, K=10, blocks=2)
    lat = lbm.Lattice.create(nx, ny, precision="f32")
    tol = 0.2
    # the identity (zero projection) on the same state: the LB's own local
    # change after the re-initialisation stays well inside the tolerance
    p["proj"] = (zero(p["proj"][0]), zero(p["proj"][1]))
    s.set_params(lbm.surrogate_params_from_oracle_layout(p))
    lat.set_fields(rho, z, z, T)
    st = s.rollout(lat, 1, drift_tol=1e-3, iface_tol=0.5, verify_steps=2, field_tol=tol)
    own = st["max_local_change_T_all"]
    assert st["accepted"] == 1 and own < 0.1 * tol, own
    A = 80.0
    wp = zero(p["proj"][0])
    for tap in range(9):
        a = 8 * A if tap == 4 else -A
        wp[tap, 3, 0], wp[tap, 3, 1] = a, -a
    p["proj"] = (wp, zero(p["proj"][1]))
    s.set_params(lbm.surrogate_params_from_oracle_layout(p))
    lat.set_fields(rho, z, z, T)
    st = s.rollout(lat, 1, drift_tol=1e-3, iface_tol=0.5, verify_steps=2, field_tol=tol)
    print("local T change: identity", own, "spike", st["max_local_change_T_all"],
          "energy drift", st["max_energy_drift_all"])
    assert st["fallbacks"] == 1 and st["accepted"] == 0 and st["unphysical"] == 0
    assert st["max_mass_drift_all"] < 1e-6 and st["max_energy_drift_all"] < 1e-3
    assert st["max_local_change_T_all"] > tol
    lat.set_fields(rho, z, z, T)
    st = s.rollout(lat, 1, drift_tol=1e-3, iface_tol=0.5, verify_steps=2, field_tol=10.0)
    assert st["accepted"] == 1
