"""Pins of the oracle's lattice Boltzmann step against identities the paper
and the mathematics fix: orthogonality of M (SM Eq. S2), the moments of the
equilibria (SM Eq. S3a, S4a with Eq. 15), the pair force on a sinusoid
(Eq. 13), exact recovery of the prescribed fields (Eq. 14), exact mass and
momentum conservation and the g budget (Eq. 12, 14), the rest state, and
the lattice symmetries (reflection, quarter turn) that a transposed entry or
flipped sign in S, L or Y would break."""
import numpy as np
import pytest

from oracle import M_and_inverse, Oracle, thermo
from paper_2106_01557_gb300 import inputs

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def random_state(n=8, seed=0, walls=0, amp_u=0.02, **kw):
    cfg = thermo.Config(nx=n, ny=n, walls=walls, **kw)
    o = Oracle(cfg)
    p = o.p
    rho = inputs.perturbed(np.full((n, n), 0.5 * (p.rho_v + p.rho_l)), 0.8, seed)
    ux, uy = inputs.random_velocity((n, n), amp_u * p.c, seed + 1)
    T = inputs.perturbed(np.full((n, n), p.T0), 0.05, seed + 2)
    o.init_fields(rho, ux, uy, T)
    # break the exact equilibrium so that every non-equilibrium term is active
    rng = np.random.default_rng(seed + 3)
    o.f *= 1.0 + 0.01 * rng.uniform(-1, 1, o.f.shape)
    o.g *= 1.0 + 0.01 * rng.uniform(-1, 1, o.g.shape)
    return o


def test_M_orthogonal_and_inverse():
    M, Mi = M_and_inverse()
    assert np.abs(M @ Mi - np.eye(9)).max() < 1e-15
    # Lallemand-Luo basis: rows mutually orthogonal with these norms
    assert np.array_equal(M @ M.T, np.diag([9.0, 36, 36, 6, 12, 6, 12, 4, 4]))
    # rows 3 and 5 are the lattice velocities (SM Eq. S1 / Eq. S2 agree)
    assert np.array_equal(M[3], EX) and np.array_equal(M[5], EY)


def test_equilibrium_velocity_terms_are_the_discrete_maxwellians():
    # At fixed rho and T (eta depends on nothing else), the velocity dependence
    # of m^eq (SM Eq. S3a) is that of the textbook second-order D2Q9
    # equilibrium w_i rho (1 + 3 e_i.u + 9/2 (e_i.u)^2 - 3/2 |u|^2) (u over the
    # lattice speed) projected with M: +3 rho |u|^2 in row e, -3 rho |u|^2 in
    # row eps (a sign no dynamic pin separates), -rho u in rows q, rho (ux^2 -
    # uy^2) and rho ux uy in rows p. The oracle's m^eq is read back from its
    # initialisation of a uniform state (no force, so f = M^-1 m^eq).
    M, _ = M_and_inverse()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    o = Oracle(thermo.Config(nx=4, ny=4))
    p = o.p
    rho0 = p.rho_v
    one = np.ones((4, 4))

    def m_eq(uxh, uyh):
        o.init_fields(rho0 * one, uxh * p.c * one, uyh * p.c * one, p.T0 * one)
        return M @ o.f[:, 1, 1]

    def maxwellian(uxh, uyh):
        eu = EX * uxh + EY * uyh
        return w * rho0 * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (uxh ** 2 + uyh ** 2))

    m0 = m_eq(0.0, 0.0)
    for uxh, uyh in [(0.1, 0.0), (0.07, -0.05), (0.0, 0.12)]:
        dm = m_eq(uxh, uyh) - m0
        dref = M @ (maxwellian(uxh, uyh) - maxwellian(0.0, 0.0))
        assert np.abs(dm - dref).max() < 1e-13 * rho0, (uxh, uyh, dm - dref)


def test_forcing_moments_are_those_of_the_second_order_forcing_term():
    # The discrete force F_m (SM Eq. S3b) is the moment projection of the
    # textbook second-order forcing term w_i [3 e_i.F + 9 (e_i.u)(e_i.F) -
    # 3 u.F] (F and u over the lattice speed): F.u enters rows e and eps as
    # +-6 F.u, the momentum rows as F, and rows p as 2 (Fx ux - Fy uy) and
    # Fx uy + Fy ux. The oracle's F_m is read back from its initialisation of a
    # uniform state with and without a body force (m = m^eq - dt/2 F_m).
    M, _ = M_and_inverse()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    one = np.ones((4, 4))
    for ax, ay, uxh, uyh in [(2e-3, 0.0, 0.1, 0.0), (1e-3, -2e-3, 0.07, -0.05), (0.0, 3e-3, 0.03, 0.11)]:
        ms = []
        for a in ((0.0, 0.0), (ax, ay)):
            o = Oracle(thermo.Config(nx=4, ny=4, accel_x=a[0], accel_y=a[1]))
            p = o.p
            o.init_fields(p.rho_v * one, uxh * p.c * one, uyh * p.c * one, p.T0 * one)
            ms.append(M @ o.f[:, 1, 1])
        Fm = 2.0 * (ms[0] - ms[1]) / p.dt
        Fxh, Fyh = p.rho_v * ax / p.c, p.rho_v * ay / p.c
        eu, eF = EX * uxh + EY * uyh, EX * Fxh + EY * Fyh
        ref = M @ (w * (3 * eF + 9 * eu * eF - 3 * (uxh * Fxh + uyh * Fyh)))
        scale = abs(Fxh) + abs(Fyh)
        assert np.abs(Fm - ref).max() < 1e-9 * scale, (ax, ay, Fm - ref)


def test_energy_source_moments_are_those_of_the_second_order_scalar_source():
    # The source q_m of the g moments (SM Eq. S4b) against the moment
    # projection of the textbook second-order source term of a scalar
    # transported by the flow, w_i q [1 + 3 e_i.u] (u over the lattice
    # speed): M of it is [q, -2 q, q, q ux, -q ux, q uy, -q uy, 0, 0]. At the
    # paper's gamma1 = -2 rows 0, 1 and 3-8 of S4b must equal these; that
    # fixes which of gamma1, gamma2 sits in row e (swapped, row e would read
    # 2 q) and the sign of the heat-flux rows. Row eps of S4b is gamma2 q, a
    # free choice of the model (the paper's gamma2 = 2 gives 2 q where the
    # textbook source has q); it is checked as written. The oracle's q_m is
    # read back from its initialisation of a uniform state with and without
    # a body force: n = n^eq - dt/2 q_m with q = F.u, and n^eq does not
    # depend on the force.
    M, _ = M_and_inverse()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    one = np.ones((4, 4))
    for ax, ay, uxh, uyh in [(2e-3, 0.0, 0.1, 0.0), (1e-3, -2e-3, 0.07, -0.05), (0.0, 3e-3, -0.03, 0.11)]:
        ns = []
        for a in ((0.0, 0.0), (ax, ay)):
            o = Oracle(thermo.Config(nx=4, ny=4, accel_x=a[0], accel_y=a[1]))
            p = o.p
            o.init_fields(p.rho_v * one, uxh * p.c * one, uyh * p.c * one, p.T0 * one)
            ns.append(M @ o.g[:, 1, 1])
        qm = 2.0 * (ns[0] - ns[1]) / p.dt
        q = p.rho_v * (ax * uxh + ay * uyh) * p.c     # F.u with F = rho a
        ref = M @ (w * q * (1 + 3 * (EX * uxh + EY * uyh)))
        assert p.gamma1 == -2.0
        rows = [0, 1, 3, 4, 5, 6, 7, 8]
        assert np.abs(qm[rows] - ref[rows]).max() < 1e-9 * abs(q), (ax, ay, qm - ref)
        assert qm[2] == pytest.approx(p.gamma2 * q, rel=1e-9)


def test_init_recovers_prescribed_fields():
    o = random_state(seed=4)
    n = o.nx
    p = o.p
    rho = inputs.perturbed(np.full((n, n), 0.1), 0.5, 11)
    ux, uy = inputs.random_velocity((n, n), 0.03 * p.c, 12)
    T = inputs.perturbed(np.full((n, n), p.T0), 0.1, 13)
    o.init_fields(rho, ux, uy, T)
    m = o.moments()
    assert np.abs(m["rho"] - rho).max() < 1e-15
    assert np.abs(m["ux"] - ux).max() < 1e-15 * p.c * 10
    assert np.abs(m["uy"] - uy).max() < 1e-15 * p.c * 10
    assert np.abs(m["T"] / T - 1).max() < 1e-13


def test_equilibrium_moments_give_the_recovered_eos():
    # On a uniform state F = 0 and f = f^eq. Its second moments must be
    # p_BE delta + rho u u with p_BE = p_EOS + a rho^2 (Eq. 15, 17, text
    # after Eq. 11), and g^eq must carry rho e_k and the enthalpy flux
    # rho h_k u with rho h_k = rho e_k + p_BE (Eq. 15).
    n = 4
    for rho0, u0, v0, Tr in [(0.02, 0.01, -0.02, 0.8), (0.3, -0.03, 0.01, 0.7), (0.15, 0.0, 0.04, 0.9)]:
        o = Oracle(thermo.Config(nx=n, ny=n))
        p = o.p
        T0 = Tr * p.Tc
        u, v = u0 * p.c, v0 * p.c
        o.init_fields(np.full((n, n), rho0), np.full((n, n), u), np.full((n, n), v), np.full((n, n), T0))
        f = o.f[:, 0, 0]
        g = o.g[:, 0, 0]
        ex, ey = p.c * EX, p.c * EY
        pBE = thermo.p_eos(rho0, T0, p.a_t, p.b_t, p.R, p.K_EOS) + p.a * rho0 ** 2
        assert f.sum() == pytest.approx(rho0, rel=1e-14)
        assert (ex * f).sum() == pytest.approx(rho0 * u, rel=1e-13, abs=1e-17)
        assert (ex * ex * f).sum() == pytest.approx(pBE + rho0 * u * u, rel=1e-12)
        assert (ey * ey * f).sum() == pytest.approx(pBE + rho0 * v * v, rel=1e-12)
        assert (ex * ey * f).sum() == pytest.approx(rho0 * u * v, rel=1e-12, abs=1e-17)
        rek = rho0 * p.cv * T0 + 0.5 * rho0 * (u * u + v * v)
        assert g.sum() == pytest.approx(rek, rel=1e-13)
        assert (ex * g).sum() == pytest.approx((rek + pBE) * u, rel=1e-12, abs=1e-18)
        assert (ey * g).sum() == pytest.approx((rek + pBE) * v, rel=1e-12, abs=1e-18)


def test_pair_force_on_sinusoid_is_exact():
    # Eq. 13 with weights 1/3 and 1/12 on rho = r0 + A sin(k x):
    # sum_i w_i rho(x + e_i) e_i = A cos(k x) sin(k) exactly (dx = 1).
    n = 32
    o = Oracle(thermo.Config(nx=n, ny=8))
    p = o.p
    k = 2 * np.pi / n * 3
    x = np.arange(n)
    rho = np.repeat((0.1 + 0.05 * np.sin(k * x))[None, :], 8, axis=0)
    o.init_fields(rho, 0 * rho, 0 * rho, 0 * rho + p.T0)
    m = o.moments()
    expect = p.G2 * rho * 0.05 * np.cos(k * x)[None, :] * np.sin(k)
    assert np.abs(m["Fpx"] - expect).max() < 1e-15 * p.G2
    assert np.abs(m["Fpy"]).max() < 1e-16 * p.G2


def test_rest_state_is_a_fixed_point():
    n = 8
    o = Oracle(thermo.Config(nx=n, ny=n))
    p = o.p
    o.init_fields(np.full((n, n), p.rho_l), np.zeros((n, n)), np.zeros((n, n)), np.full((n, n), p.T0))
    f0, g0 = o.f.copy(), o.g.copy()
    o.step(50)
    assert np.abs(o.f - f0).max() < 1e-14 * np.abs(f0).max()
    assert np.abs(o.g - g0).max() < 1e-14 * np.abs(g0).max()


def test_uniform_flow_is_a_fixed_point():
    n = 8
    o = Oracle(thermo.Config(nx=n, ny=n))
    p = o.p
    o.init_fields(np.full((n, n), p.rho_v), np.full((n, n), 0.02 * p.c), np.full((n, n), -0.01 * p.c),
                  np.full((n, n), p.T0))
    f0 = o.f.copy()
    o.step(20)
    assert np.abs(o.f - f0).max() < 1e-14 * np.abs(f0).max()


def test_exact_conservation_on_periodic_box():
    o = random_state(seed=7)
    p = o.p
    c0 = o.conservation()
    m0 = o.moments()
    sum_g0 = o.g.sum()
    q0 = m0["q"].sum()
    o.step(1)
    c1 = o.conservation()
    # mass: F_m[0] = 0 and the rho row of m - m^eq vanishes
    assert c1[0] == pytest.approx(c0[0], rel=1e-14)
    # momentum: sum of F_pair cancels pairwise; no body force
    scale = c0[0] * p.c
    assert abs(c1[1] - c0[1]) < 1e-14 * scale
    assert abs(c1[2] - c0[2]) < 1e-14 * scale
    # g budget: sum g^{n+1} = sum g^n + dt sum q^n (row 0 of Eq. 12c)
    assert o.g.sum() == pytest.approx(sum_g0 + p.dt * q0, rel=1e-14)
    o.step(20)
    c2 = o.conservation()
    assert c2[0] == pytest.approx(c0[0], rel=1e-13)
    assert abs(c2[1] - c0[1]) < 1e-13 * scale


def test_body_force_momentum_budget():
    o = random_state(seed=9, accel_x=1e-4, accel_y=-2e-4)
    p = o.p
    c0 = o.conservation()
    o.step(3)
    c1 = o.conservation()
    assert c1[1] - c0[1] == pytest.approx(3 * p.dt * c0[0] * 1e-4, rel=1e-10)
    assert c1[2] - c0[2] == pytest.approx(-3 * p.dt * c0[0] * 2e-4, rel=1e-10)


def _rotate(a):
    """Quarter turn of a population array (9, n, n): position (x, y) ->
    (-y, x), direction (ex, ey) -> (-ey, ex)."""
    perm = {0: 0, 1: 2, 2: 3, 3: 4, 4: 1, 5: 6, 6: 7, 7: 8, 8: 5}
    out = np.empty_like(a)
    for i, j in perm.items():
        # new[y', x'] with x' = -y, y' = x  ->  new = rot90 of the plane
        out[j] = np.rot90(a[i], k=1, axes=(1, 0))
    return out


def _mirror(a):
    """Reflection x -> -x: (ex, ey) -> (-ex, ey)."""
    perm = {0: 0, 1: 3, 2: 2, 3: 1, 4: 4, 5: 6, 6: 5, 7: 8, 8: 7}
    out = np.empty_like(a)
    for i, j in perm.items():
        out[j] = np.roll(a[i][:, ::-1], 1, axis=1)
    return out


@pytest.mark.parametrize("sym", ["rotate", "mirror"])
def test_step_commutes_with_lattice_symmetries(sym):
    T = _rotate if sym == "rotate" else _mirror
    a = random_state(n=8, seed=21)
    b = Oracle(a.cfg, a.p)
    b.set_populations(T(a.f), T(a.g))
    a.step(3)
    b.step(3)
    assert np.abs(T(a.f) - b.f).max() < 1e-14 * np.abs(a.f).max()
    assert np.abs(T(a.g) - b.g).max() < 1e-14 * np.abs(a.g).max()


def test_single_node_collision_budget():
    # Eq. 12b, 12c at one node: mass unchanged, momentum advanced by dt F,
    # energy moment advanced by dt q.
    o = random_state(seed=3)
    p = o.p
    rng = np.random.default_rng(5)
    fl = o.f[:, 2, 3].copy()
    gl = o.g[:, 2, 3].copy()
    rho_nb = fl.sum() * (1 + 0.2 * rng.uniform(-1, 1, 9))
    fb, gb, macro = o.collide_node(fl, gl, rho_nb)
    rho, ux, uy, T, Fx, Fy, q, rek = macro
    assert fb.sum() == pytest.approx(fl.sum(), rel=1e-15)
    assert p.c * (EX * fb).sum() == pytest.approx(p.c * (EX * fl).sum() + p.dt * Fx, rel=1e-13)
    assert p.c * (EY * fb).sum() == pytest.approx(p.c * (EY * fl).sum() + p.dt * Fy, rel=1e-13)
    assert gb.sum() == pytest.approx(gl.sum() + p.dt * q, rel=1e-14)


def _linearised_step(o, rho0, ux=0.0, uy=0.0):
    """The step linearised around the uniform state at density rho0, moving
    at (ux, uy) c_s: collision Jacobian by central differences of the
    oracle's node collision, pair force through the neighbour densities,
    streaming as a phase. Returns (kx, ky) -> the 18 x 18 amplification
    matrix of the Fourier mode exp(i(kx x + ky y)) of (f, g). With the
    cubic-term elimination on, the collision also reads the central
    differences d_x(rho u_x^3), d_y(rho u_y^3) (u over c), whose mode is a
    linear function of the node's own f: d(rho u^3) = 3 u^2 d(rho u) - 2 u^3
    d(rho), rho u including dt/2 of the pair force, and a central
    difference is i sin(k)."""
    p = o.p
    n = 4
    o.init_fields(np.full((n, n), rho0), np.full((n, n), ux * p.cs), np.full((n, n), uy * p.cs),
                  np.full((n, n), p.T0))
    cubic = bool(getattr(p, "cubic", 0))
    nin = 29 if cubic else 27
    x0 = np.concatenate([o.f[:, 0, 0], o.g[:, 0, 0], np.full(9, rho0)] + ([np.zeros(2)] if cubic else []))

    def col(x):
        fb, gb, _ = o.collide_node(x[:9], x[9:18], x[18:27], x[27:29] if cubic else None)
        return np.concatenate([fb, gb])

    J = np.zeros((18, nin))
    for j in range(nin):
        h = 1e-6 * max(abs(x0[j]), 1e-3)
        xp, xm = x0.copy(), x0.copy()
        xp[j] += h
        xm[j] -= h
        J[:, j] = (col(xp) - col(xm)) / (2 * h)
    sel = np.concatenate([np.ones(9), np.zeros(9)])
    w = np.array([0] + [1 / 3] * 4 + [1 / 12] * 4)
    uxh, uyh = ux * p.cs / p.c, uy * p.cs / p.c

    def amplification(kx, ky):
        ph = np.exp(1j * (kx * EX + ky * EY))
        A = J[:, :18].astype(complex) + np.outer(J[:, 18:27] @ ph, sel)
        if cubic:
            # the pair force of the mode, over c and per unit d(rho)
            dF = p.G2 / p.c * rho0 * np.array([(w * EX * ph).sum(), (w * EY * ph).sum()])
            rows = []
            for e, u0, d, k in ((EX, uxh, 0, kx), (EY, uyh, 1, ky)):
                dj = e.astype(complex) + 0.5 * p.dt * dF[d]         # d(rho u) per d f_i
                dphi = 3 * u0 * u0 * dj - 2 * u0 ** 3                # d(rho u^3) per d f_i
                rows.append(1j * np.sin(k) * dphi)
            B = np.zeros((2, 18), dtype=complex)
            B[:, :9] = np.array(rows)
            A = A + J[:, 27:29] @ B
        P = np.diag(np.concatenate([np.conj(ph), np.conj(ph)]))
        return P @ A

    return amplification


def _growth(o, rho0, ngrid=10, U=0.0):
    """Largest amplification factor of the linearised step over a grid of
    wave vectors, around the uniform state at density rho0 moving along x at
    U c_s (at rest for U = 0)."""
    amplification = _linearised_step(o, rho0, ux=U)
    worst = 0.0
    for kx in np.linspace(0, np.pi, ngrid):
        for ky in np.linspace(0, np.pi, ngrid):
            worst = max(worst, np.abs(np.linalg.eigvals(amplification(kx, ky))).max())
    return worst


@pytest.mark.parametrize("Tr", [0.75, 0.8, 0.95])
def test_bulk_phases_linearly_stable(Tr):
    # with the default rates both bulk phases are linearly stable for
    # T_r >= 0.75 (the paper's runs use 0.8 and 0.85)
    o = Oracle(thermo.Config(nx=4, ny=4, Tr0=Tr))
    assert _growth(o, o.p.rho_l) < 1 + 1e-7
    assert _growth(o, o.p.rho_v) < 1 + 1e-7


def test_moving_vapour_linearly_stable():
    # the uniform vapour at T_r = 0.8 moving at 0.1 and 0.2 c_s stays linearly
    # stable with the coupling k s_eps omega_e of S (row e, column eps; SM
    # Eq. S5a); dropping that coefficient (growth 1e-3 at 0.1 c_s), halving
    # it (3e-4 at 0.2 c_s), doubling it (0.31 at rest) or flipping its sign
    # (0.05 at rest) makes it unstable
    o = Oracle(thermo.Config(nx=4, ny=4))
    for U in (0.0, 0.1, 0.2):
        assert _growth(o, o.p.rho_v, U=U) < 1 + 1e-7, U


def _sound_decay_asymmetry(o, rho0, U, k, along_x):
    """(d_down - d_up) / (d_down + d_up) for the two sound modes of wave
    number k travelling along the flow of the uniform state at density rho0
    moving at U c_s (along x or y): d = -ln|lambda| per step, the modes being
    the two hydrodynamic eigenvalues of the linearised step whose phases,
    with the Doppler phase k U c_s dt taken off, are the extremes."""
    amplification = _linearised_step(o, rho0, ux=U if along_x else 0.0, uy=0.0 if along_x else U)
    ev = np.linalg.eigvals(amplification(k, 0.0) if along_x else amplification(0.0, k))
    hyd = ev[np.abs(ev) > 0.8] * np.exp(1j * k * U * o.p.cs * o.p.dt)
    down, up = hyd[np.argmin(np.angle(hyd))], hyd[np.argmax(np.angle(hyd))]
    d_down, d_up = -np.log(abs(down)), -np.log(abs(up))
    return (d_down - d_up) / (d_down + d_up)


def test_sound_decays_alike_up_and_down_a_moving_vapour():
    # Galilean invariance of the normal stress (Eq. 6b): in the frame of a
    # uniform flow, sound going down- and upstream decays alike. Pins the
    # velocity couplings of S in row e (SM Eq. S5a): h u_x s_q omega_e acts on
    # waves along x in a flow along x, h u_y s_q omega_e along y. Vapour at
    # 0.05 c_s, wavelength 64: measured 1.2e-4 (the residual grows as U^3:
    # 2.1e-2 at 0.2 c_s, the D2Q9 lattice's missing cubic moments); dropping
    # the coupling gives 1.9e-2, linear in U
    o = Oracle(thermo.Config(nx=4, ny=4))
    for along_x in (True, False):
        assert abs(_sound_decay_asymmetry(o, o.p.rho_v, 0.05, 2 * np.pi / 64, along_x)) < 2e-3, along_x


def test_moving_liquid_stability_limit():
    # with the default rates the uniform liquid is linearly stable at rest
    # but not in motion: at T_r = 0.8 it grows above about 0.034 c_s (0.012
    # at T_r = 0.75, 0.093 at 0.9; the vapour holds to 0.2 c_s), a thermal
    # mode, as the rates of g move the limit most. Two rates of g that the
    # paper leaves free, sigma_eps = 1.4 and sigma_p = 1.8, keep both phases
    # stable at rest down to T_r = 0.65 (the defaults: 0.75) and the moving
    # liquid to 0.157 c_s at T_r = 0.8 (0.106 at 0.75, 0.074 at 0.7)
    o = Oracle(thermo.Config(nx=4, ny=4))
    assert _growth(o, o.p.rho_l, ngrid=20, U=0.03) < 1 + 1e-7
    assert _growth(o, o.p.rho_l, ngrid=20, U=0.05) > 1 + 1e-3
    for Tr in (0.65, 0.8):
        o = Oracle(thermo.Config(nx=4, ny=4, Tr0=Tr, sig_eps=1.4, sig_p=1.8))
        for rho0 in (o.p.rho_l, o.p.rho_v):
            assert _growth(o, rho0, ngrid=20) < 1 + 1e-7, Tr
    assert _growth(o, o.p.rho_l, ngrid=20, U=0.12) < 1 + 1e-7


def test_bulk_liquid_unstable_at_low_temperature():
    # the same rates leave the dense liquid linearly unstable at T_r = 0.6
    # (2% per step, fastest near the grid scale; below T_r = 0.75 a band of
    # short waves grows), the reason the sweep's temperatures start at 0.75
    o = Oracle(thermo.Config(nx=4, ny=4, Tr0=0.6))
    assert _growth(o, o.p.rho_l) > 1.01


def test_strip_reference_reproduces_the_full_lattice():
    # the periodic-crop reference that the full-size GPU parity test uses,
    # checked against the oracle on the whole lattice: walls, body force and a
    # hot wall segment that the strips cut at either end, and a strip across
    # the periodic seam
    from gpu_common import boiling_fields, strip_reference
    cfg = dict(nx=192, ny=40, walls=1, accel_y=-1e-5, Tr_bottom=0.8, Tr_hot=0.95, hot_x0=100, hot_len=32)
    o = Oracle(thermo.Config(**cfg))
    fields = boiling_fields(192, 40, o.p, seed=21)
    o.init_fields(*fields)
    o.step(10)
    full = o.moments()
    for x0 in (80, 120, 0, 170):
        ref = strip_reference(fields, cfg, x0, 48, 24, 10)
        for k in ("rho", "ux", "uy", "T"):
            got = np.roll(full[k], -x0, axis=1)[:, :48]
            assert np.abs(got - ref[k]).max() <= 1e-12 * np.abs(full[k]).max(), (x0, k)


def test_cubic_terms_third_moments_of_the_equilibrium():
    # The cubic-term elimination (paragraph after Eq. 16; a reading, the
    # details being in another paper): the equilibria of q_x, q_y gain
    # 3 rho u_x u_y^2 and 3 rho u_y u_x^2 (u over c), so that the lattice
    # third moments Q_xyy = sum e_x e_y^2 f and Q_xxy of the equilibrium are
    # those of the continuous Maxwellian, rho u_x / 3 + rho u_x u_y^2 and
    # rho u_y / 3 + rho u_x^2 u_y (over c^3); without it the cubic parts are
    # missing. Read back from the initialisation of a uniform state.
    one = np.ones((4, 4))
    for uxh, uyh in [(0.1, 0.07), (-0.05, 0.12)]:
        for cubic in (0, 1):
            o = Oracle(thermo.Config(nx=4, ny=4, cubic=cubic))
            p = o.p
            o.init_fields(p.rho_v * one, uxh * p.c * one, uyh * p.c * one, p.T0 * one)
            f = o.f[:, 1, 1]
            qxyy = (EX * EY * EY * f).sum()
            qxxy = (EX * EX * EY * f).sum()
            cub = (p.rho_v * uxh * uyh * uyh, p.rho_v * uxh * uxh * uyh) if cubic else (0.0, 0.0)
            assert qxyy == pytest.approx(p.rho_v * uxh / 3 + cub[0], rel=1e-12)
            assert qxxy == pytest.approx(p.rho_v * uyh / 3 + cub[1], rel=1e-12)


def test_cubic_source_cancels_most_of_the_u3_sound_asymmetry():
    # The D2Q9 lattice cannot carry the rho u_x^3 of Q_xxx; the elimination's
    # source -c d_x(rho u_x^3) in the deviatoric stress makes it up. Sound
    # going down- and upstream of a moving vapour (wavelength 64) decays
    # alike up to an error a U + b U^3: uncorrected 9.3e-3 U - 2.76 U^3
    # (-2.1e-2 at 0.2 c_s); with the source the U^3 part falls to -0.42 U^3
    # (-1.5e-3 at 0.2 c_s), and the linear part, which is not a cubic term,
    # stays. The flipped source doubles the error (-5.5e-2), and putting the
    # source into the trace row e as well over-corrects (+8.3e-3).
    for cubic, lo, hi in ((0, -2.3e-2, -1.9e-2), (1, -2.5e-3, -0.5e-3)):
        o = Oracle(thermo.Config(nx=4, ny=4, cubic=cubic))
        for along_x in (True, False):
            a = _sound_decay_asymmetry(o, o.p.rho_v, 0.2, 2 * np.pi / 64, along_x)
            assert lo < a < hi, (cubic, along_x, a)
        # and it stays linearly stable, moving and at rest
        assert _growth(o, o.p.rho_v, U=0.2) < 1 + 1e-7
        assert _growth(o, o.p.rho_l) < 1 + 1e-7


def test_cubic_terms_keep_the_step_invariants():
    # with the elimination on: mass and momentum exact on a periodic box,
    # and a uniform flow stays a fixed point (the source is a difference of
    # neighbours' values)
    o = random_state(seed=31, cubic=1)
    p = o.p
    c0 = o.conservation()
    o.step(5)
    c1 = o.conservation()
    assert c1[0] == pytest.approx(c0[0], rel=1e-14)
    assert abs(c1[1] - c0[1]) < 1e-13 * c0[0] * p.c and abs(c1[2] - c0[2]) < 1e-13 * c0[0] * p.c
    n = 8
    o = Oracle(thermo.Config(nx=n, ny=n, cubic=1))
    p = o.p
    o.init_fields(np.full((n, n), p.rho_v), np.full((n, n), 0.05 * p.c), np.full((n, n), -0.03 * p.c),
                  np.full((n, n), p.T0))
    f0 = o.f.copy()
    o.step(20)
    assert np.abs(o.f - f0).max() < 1e-14 * np.abs(f0).max()


def test_cubic_terms_of_the_full_step_agree_with_the_linearised_step():
    # The full step computes rho u^3 at every node and differences it; the
    # linearised step forms the same from the Fourier mode. A small density
    # wave (k = 2 pi / 16) on a vapour moving at 0.2 c_s: the change the
    # cubic-term elimination makes to the wave's (f, g) amplitude in one step
    # must be the same in both, to the wave's small amplitude (a dropped
    # neighbour, a wrong index or u in place of u / c in the full step's
    # rho u^3 fails this).
    n, k, eps = 16, 2 * np.pi / 16, 1e-6
    x = np.arange(n)
    amps = {}
    for cubic in (0, 1):
        o = Oracle(thermo.Config(nx=n, ny=4, cubic=cubic))
        p = o.p
        U = 0.2 * p.cs
        one = np.ones((4, n))
        o.init_fields(p.rho_v * one, U * one, 0 * one, p.T0 * one)
        fb, gb = o.f.copy(), o.g.copy()
        o.init_fields(p.rho_v * (1 + eps * np.cos(k * x))[None, :] * one, U * one, 0 * one, p.T0 * one)
        d0 = np.concatenate([o.f - fb, o.g - gb])[:, 0, :]          # (18, n)
        a0 = (d0 * np.exp(-1j * k * x)).sum(axis=1) / n
        o.step(1)
        d1 = np.concatenate([o.f - fb, o.g - gb])[:, 0, :]
        a1 = (d1 * np.exp(-1j * k * x)).sum(axis=1) / n
        amp = _linearised_step(Oracle(thermo.Config(nx=4, ny=4, cubic=cubic)), p.rho_v, ux=0.2)
        amps[cubic] = (a1, amp(k, 0.0) @ a0)
    d_full = amps[1][0] - amps[0][0]
    d_lin = amps[1][1] - amps[0][1]
    assert np.abs(d_lin).max() > 1e-5 * np.abs(amps[0][1]).max()     # the terms act (8e-5 of the wave)
    assert np.abs(d_full - d_lin).max() < 1e-3 * np.abs(d_lin).max(), np.abs(d_full - d_lin).max() / np.abs(d_lin).max()
