"""Pins of the spin-polarised oracle (oracle/spin.py) against what is fixed
outside it: the unpolarised oracle (itself pinned to the appendix and to
Dion's screened-exchange form), the spin-scaling identity of exchange
evaluated through the unpolarised q0, PW92's high-density structure and the
definition of its spin interpolation, symmetry, and finite differences."""
import numpy as np
import pytest

from oracle import spin, vdw


# ---------------------------------------------------------------------------
# PW92 correlation with spin interpolation
# ---------------------------------------------------------------------------
def test_pw92_spin_endpoints():
    rs = np.geomspace(0.05, 80.0, 40)
    e0, d0 = vdw.pw92_eps_c(rs)
    e, drs, dz = spin.pw92_eps_c_spin(rs, np.zeros_like(rs))
    assert np.array_equal(e, e0) and np.allclose(drs, d0, rtol=1e-14, atol=0)
    assert np.max(np.abs(dz)) == 0.0                      # f'(0) = 0: stationary at zeta = 0
    e1, _ = spin.pw92_G(rs, spin.PW92_P1)
    for z in (1.0, -1.0):
        ez, _, _ = spin.pw92_eps_c_spin(rs, np.full_like(rs, z))
        assert np.allclose(ez, e1, rtol=1e-14, atol=0)
    f, df = spin.f_zeta(np.array([0.0, 1.0, -1.0]))
    assert np.allclose(f, [0.0, 1.0, 1.0], atol=1e-15) and df[0] == 0.0
    # a polarised gas has less correlation energy per particle, monotonically in |zeta|
    ez = [spin.pw92_eps_c_spin(rs, np.full_like(rs, z))[0] for z in (0.0, 0.3, 0.6, 0.9, 1.0)]
    assert all(np.all(a < b) for a, b in zip(ez, ez[1:]))


def test_pw92_fz20_is_the_second_derivative_of_f():
    exact = (8.0 / 9.0) / (2.0 ** (4.0 / 3.0) - 2.0)
    assert abs(spin.FZ20 - exact) <= 1e-6 * exact
    h = 1e-3
    f = spin.f_zeta(np.array([-h, 0.0, h]))[0]
    assert abs((f[0] - 2 * f[1] + f[2]) / h ** 2 - exact) <= 1e-5 * exact


@pytest.mark.parametrize("par,A_exact,c1", [
    (spin.PW92_P0, (1.0 - np.log(2.0)) / np.pi ** 2, 0.046644),          # paramagnetic
    (spin.PW92_P1, (1.0 - np.log(2.0)) / (2.0 * np.pi ** 2), 0.025599),  # ferromagnetic
    (spin.PW92_PA, 1.0 / (6.0 * np.pi ** 2), 0.035475),                 # -alpha_c
])
def test_pw92_parameters_follow_the_high_density_expansion(par, A_exact, c1):
    # eps -> A ln r_s - c1 + ... as r_s -> 0 fixes A (the RPA log coefficient:
    # (1 - ln 2)/pi^2, half of it when fully polarised, 1/(6 pi^2) for the spin
    # stiffness), beta1 = exp(-c1 / 2A) / 2A and beta2 = 2 A beta1^2
    A, a1, b1, b2, b3, b4 = par
    assert abs(A - A_exact) <= 3e-5 * A_exact
    assert abs(b1 - np.exp(-c1 / (2 * A)) / (2 * A)) <= 1e-4 * b1
    assert abs(b2 - 2 * A * b1 * b1) <= 1e-4 * b2
    rs = 1e-7
    g, _ = spin.pw92_G(np.array([rs]), par)
    assert abs(g[0] - (A * np.log(rs) - c1)) < 2e-3


# ---------------------------------------------------------------------------
# Spin q0
# ---------------------------------------------------------------------------
def _inputs(seed=0, k=400):
    g = np.random.default_rng(seed)
    n = 10 ** g.uniform(-6, 0.5, k)
    zeta = g.uniform(-0.95, 0.95, k)
    nu, nd = n * (1 + zeta) / 2, n * (1 - zeta) / 2
    su = (nu ** (4 / 3)) ** 2 * 10 ** g.uniform(-3, 1.5, k)
    sd = (nd ** (4 / 3)) ** 2 * 10 ** g.uniform(-3, 1.5, k)
    return nu, nd, su, sd


@pytest.mark.parametrize("functional", [1, 2])
def test_spin_q0_unpolarised_limit_is_the_appendix_q0(functional):
    g = np.random.default_rng(3)
    n = np.concatenate([10 ** g.uniform(-7, 1, 300), [1e-13, 0.0, 5e-12, 50.0]])
    s = np.concatenate([n[:300] ** (8 / 3) * 10 ** g.uniform(-4, 2, 300), [0.0, 0.0, 1e-30, 1e3]])
    q, dn, ds = vdw.q0_of(n, s, functional)
    qs, d, live = spin.q0_spin(n / 2, n / 2, s / 4, s / 4, functional)
    assert np.array_equal(live, n > vdw.Params().n_min)
    assert np.allclose(qs, q, rtol=1e-14, atol=0)
    # sigma fixed, n_up = n_dn = n / 2: dq0/dn = (dq0/dn_up + dq0/dn_dn) / 2, and
    # the two are equal; sigma_ss = sigma / 4 for both: dq0/dsigma = (d_upup + d_dndn) / 4
    scale_n = np.maximum(np.abs(dn), 1e-300)
    assert np.max(np.abs(d[0] - dn) / scale_n) < 1e-12 and np.max(np.abs(d[1] - dn) / scale_n) < 1e-12
    assert np.allclose(d[2], 2 * ds, rtol=1e-13, atol=0) and np.allclose(d[3], 2 * ds, rtol=1e-13, atol=0)


def _h_inverse(q0, a):
    lo, hi = np.zeros_like(q0), np.full_like(q0, 3.0 * a)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        up = vdw.saturate(mid, a)[0] > q0
        hi = np.where(up, mid, hi)
        lo = np.where(up, lo, mid)
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("functional", [1, 2])
def test_spin_exchange_obeys_spin_scaling_through_the_unpolarised_q0(functional):
    # E_x[n_up, n_dn] = (E_x[2 n_up] + E_x[2 n_dn]) / 2 per particle:
    # x(n_up, n_dn) = sum_s (n_s / n) x_unpol(2 n_s, |2 grad n_s|^2).  x_unpol is
    # taken from the unpolarised q0 by undoing its saturation and its
    # correlation: x_unpol(m, s) = h^-1(q0(m, s)) + (4 pi / 3) eps_c(r_s(m)).
    p = vdw.Params()
    g = np.random.default_rng(7 + functional)
    k = 200
    n = 10 ** g.uniform(-4, -1.5, k)
    zeta = g.uniform(-0.9, 0.9, k)
    nu, nd = n * (1 + zeta) / 2, n * (1 - zeta) / 2
    su = nu ** (8 / 3) * 10 ** g.uniform(-2, 0.5, k)
    sd = nd ** (8 / 3) * 10 ** g.uniform(-2, 0.5, k)

    def x_unpol(m, s):
        q0, _, _ = vdw.q0_of(m, s, functional, p)
        assert np.all(q0 > p.q_min) and np.all(q0 < 0.8 * p.q_cut)
        rs = np.cbrt(3.0 / (4.0 * np.pi * m))
        return _h_inverse(q0, p.q_cut) + (4.0 * np.pi / 3.0) * vdw.pw92_eps_c(rs)[0]

    expect = (nu / n) * x_unpol(2 * nu, 4 * su) + (nd / n) * x_unpol(2 * nd, 4 * sd)
    _, _, xsum, _ = spin.q_raw_spin(nu, nd, su, sd, functional, p)
    assert np.max(np.abs(xsum - expect) / np.abs(expect)) < 1e-11


def test_spin_q0_derivatives_match_finite_differences():
    nu, nd, su, sd = _inputs(1, 200)
    base = [nu, nd, su, sd]
    qr, dr, _, _ = spin.q_raw_spin(*base, 2)
    q0, d, _ = spin.q0_spin(*base, 2)
    ok = (q0 > 1e-3) & (q0 < 3.0)                         # away from the clamp and deep saturation
    assert ok.sum() > 50
    for i in range(4):
        h = 1e-6 * base[i]
        up = list(base)
        dn = list(base)
        up[i] = base[i] + h
        dn[i] = base[i] - h
        # q_raw everywhere (smooth), q0 where the saturation is well conditioned
        # (tolerance: truncation plus the rounding of q_raw over the step)
        fd = (spin.q_raw_spin(*up, 2)[0] - spin.q_raw_spin(*dn, 2)[0]) / (2 * h)
        tol = 1e-7 * np.abs(dr[i]) + 1e-15 * np.abs(qr) / h
        assert np.all(np.abs(fd - dr[i]) <= tol), i
        fd = (spin.q0_spin(*up, 2)[0] - spin.q0_spin(*dn, 2)[0]) / (2 * h)
        tol = 1e-6 * np.abs(d[i]) + 2e-14 * np.abs(qr) / h      # saturation adds a few ulps
        assert np.all((np.abs(fd - d[i]) <= tol)[ok]), i


def test_spin_q0_swaps_with_the_spins_and_dead_channels_are_finite():
    nu, nd, su, sd = _inputs(2, 100)
    q, d, _ = spin.q0_spin(nu, nd, su, sd, 1)
    qs, ds, _ = spin.q0_spin(nd, nu, sd, su, 1)
    assert np.allclose(q, qs, rtol=1e-14, atol=0)
    for a, b in ((0, 1), (1, 0), (2, 3), (3, 2)):
        assert np.allclose(d[a], ds[b], rtol=1e-12, atol=0)
    # fully polarised points (one channel empty) and negative inputs
    z = np.zeros(4)
    q, d, live = spin.q0_spin(np.array([0.01, 0.1, 1e-13, -1e-3]), z, np.array([1e-5, 1e-3, 0.0, 1.0]),
                              np.array([3.0, 0.0, 0.0, -1.0]), 1)
    assert np.all(np.isfinite(q)) and all(np.all(np.isfinite(x)) for x in d)
    assert list(live) == [True, True, False, False]
    assert np.all(d[3] == 0.0)                            # the empty channel's sigma does not enter
    # the fully polarised point is the limit of nearly polarised ones
    qe, de, _ = spin.q0_spin(np.array([0.01]), np.array([1e-11]), np.array([1e-5]), np.array([0.0]), 1)
    assert abs(qe[0] - q[0]) < 1e-6 * q[0]


# ---------------------------------------------------------------------------
# Energy and potentials on a grid
# ---------------------------------------------------------------------------
def _grid_system(shape=(10, 10, 12), seed=5):
    from paper_1703_06999_gb300 import inputs
    g = np.random.default_rng(seed)
    L = np.array(shape) * 0.5
    cell = np.array([[L[0], 0, 0], [0.4, L[1], 0], [-0.3, 0.2, L[2]]])
    atoms = [(float(g.uniform(1, 4)), float(g.uniform(1, 2)), tuple(g.uniform(0, 1, 3) @ cell)) for _ in range(3)]
    s = inputs.make_system(shape, cell, atoms, 2)
    n = s.n.numpy()
    x = np.arange(shape[0])[:, None, None] / shape[0]
    zeta = 0.6 * np.sin(2 * np.pi * x) * np.ones(shape)     # a smooth spin texture
    nu, nd = n * (1 + zeta) / 2, n * (1 - zeta) / 2
    return s, nu, nd


def test_spin_energy_unpolarised_limit(oracle_default):
    s, _, _ = _grid_system()
    n, sg = s.n.numpy(), s.sigma.numpy()
    ref = oracle_default.energy_potential(n, sg, s.cell, s.functional)
    e, dn, ds = spin.energy_potential_spin(oracle_default, n / 2, n / 2, sg / 4, sg / 4, s.cell, s.functional)
    assert abs(e - ref.energy) <= 1e-13 * abs(ref.energy)
    for x in dn:
        assert np.max(np.abs(x - ref.dedn)) <= 1e-12 * np.max(np.abs(ref.dedn))
    for x in ds:
        assert np.max(np.abs(x - 2 * ref.dedsigma)) <= 1e-12 * np.max(np.abs(ref.dedsigma))


def test_spin_potentials_are_derivatives_of_the_energy(oracle_default):
    s, nu, nd = _grid_system((8, 8, 10), 6)
    g = np.random.default_rng(9)
    su = nu ** (8 / 3) * g.uniform(0.1, 2.0, nu.shape)
    sd = nd ** (8 / 3) * g.uniform(0.1, 2.0, nd.shape)
    args = [nu, nd, su, sd]
    e, dn, ds = spin.energy_potential_spin(oracle_default, *args, s.cell, s.functional)
    dV = vdw.cell_volume(s.cell) / nu.size
    pots = list(dn) + list(ds)
    idx = np.argmax(nu)                                    # a point of high density
    for i in range(4):
        for j in (idx, idx // 3):
            a = args[i].ravel()[j]
            h = 1e-4 * a
            up = [x.copy() for x in args]
            dnl = [x.copy() for x in args]
            up[i].flat[j] = a + h
            dnl[i].flat[j] = a - h
            ep = spin.energy_potential_spin(oracle_default, *up, s.cell, s.functional)[0]
            em = spin.energy_potential_spin(oracle_default, *dnl, s.cell, s.functional)[0]
            fd = (ep - em) / (2 * h)
            an = dV * pots[i].ravel()[j]
            assert abs(fd - an) <= 1e-5 * max(abs(an), abs(fd)) + 1e-14, (i, j, fd, an)


def test_spin_energy_swaps_with_the_spins(oracle_default):
    s, nu, nd = _grid_system((8, 10, 8), 8)
    su, sd = 0.3 * nu ** (8 / 3), 1.7 * nd ** (8 / 3)
    e, dn, ds = spin.energy_potential_spin(oracle_default, nu, nd, su, sd, s.cell, s.functional)
    e2, dn2, ds2 = spin.energy_potential_spin(oracle_default, nd, nu, sd, su, s.cell, s.functional)
    assert abs(e - e2) <= 1e-13 * abs(e)
    assert np.allclose(dn[0], dn2[1], rtol=1e-10, atol=1e-14) and np.allclose(ds[1], ds2[0], rtol=1e-10, atol=1e-14)
