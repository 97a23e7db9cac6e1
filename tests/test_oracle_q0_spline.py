"""Pins of the oracle's q0(n, sigma), saturation and helper splines."""
import numpy as np
import pytest

from oracle import vdw


def test_pw92_high_density_log_coefficient():
    # Exact RPA high-density limit (Gell-Mann--Brueckner): eps_c ~ c0 ln r_s
    # with c0 = (1 - ln 2) / pi^2; PW92's A is that coefficient.
    rs = np.array([1e-6, 2e-6])
    eps, _ = vdw.pw92_eps_c(rs)
    slope = (eps[1] - eps[0]) / np.log(2.0)
    assert slope == pytest.approx((1 - np.log(2)) / np.pi ** 2, rel=2e-3)


@pytest.mark.parametrize("rs,val", [(1.0, -0.0598), (2.0, -0.0448)])
def test_pw92_reference_values(rs, val):
    # Correlation energy per particle of the uniform gas (QMC fit), Hartree.
    eps, _ = vdw.pw92_eps_c(np.array([rs]))
    assert eps[0] == pytest.approx(val, rel=5e-3)


def test_pw92_derivative_fd():
    rs = np.array([0.3, 1.0, 4.0, 20.0])
    h = 1e-6 * rs
    e1, _ = vdw.pw92_eps_c(rs + h)
    e0, _ = vdw.pw92_eps_c(rs - h)
    _, d = vdw.pw92_eps_c(rs)
    assert np.allclose(d, (e1 - e0) / (2 * h), rtol=1e-7)


def test_saturation_identity_small_x_and_limit():
    x = np.linspace(0.0, 0.5, 51)
    h, dh = vdw.saturate(x, 5.0)
    # sum_{m>=1} t^m / m = -ln(1 - t) => h = x up to the t^13 tail
    assert np.max(np.abs(h - x)) < 1e-12
    assert np.allclose(dh, 1.0, atol=1e-11)
    big = np.array([5.0, 10.0, 50.0, 1e3])
    hb, _ = vdw.saturate(big, 5.0)
    assert np.all(hb < 5.0 + 1e-15) and np.all(np.diff(hb) >= 0)
    assert hb[-1] == pytest.approx(5.0, abs=1e-15)


def test_saturation_derivative_fd():
    x = np.array([0.5, 2.0, 4.0, 6.0, 9.0])
    e = 1e-6
    h1, _ = vdw.saturate(x + e, 5.0)
    h0, _ = vdw.saturate(x - e, 5.0)
    _, dh = vdw.saturate(x, 5.0)
    assert np.allclose(dh, (h1 - h0) / (2 * e), rtol=1e-6, atol=1e-12)


def test_q0_uniform_gas_kF_rs_relation():
    # For sigma = 0 and small q0 (no saturation, h(x) ~ x), q0 = k_F - (4 pi/3) eps_c(r_s)
    # with k_F r_s = (9 pi / 4)^{1/3}: pins the reading of the garbled r_s relation.
    n = np.array([1e-5, 1e-4])
    q0, _, _ = vdw.q0_of(n, np.zeros(2), vdw.DF1)
    kF = (3 * np.pi ** 2 * n) ** (1 / 3)
    rs = (9 * np.pi / 4) ** (1 / 3) / kF
    eps, _ = vdw.pw92_eps_c(rs)
    want, _ = vdw.saturate(kF - 4 * np.pi / 3 * eps, 5.0)
    assert np.allclose(q0, want, rtol=1e-13)
    # and the printed r_s^3 = 4 pi n / 3 reading would give a different q0
    rs_bad = (4 * np.pi * n / 3) ** (1 / 3)
    eps_bad, _ = vdw.pw92_eps_c(rs_bad)
    bad, _ = vdw.saturate(kF - 4 * np.pi / 3 * eps_bad, 5.0)
    assert np.all(np.abs(bad / q0 - 1) > 1e-2)


def test_q0_derivatives_fd():
    rng = np.random.default_rng(0)
    n = 10 ** rng.uniform(-4, 0.5, 40)
    s = 10 ** rng.uniform(-6, 0, 40) * n ** (8 / 3)
    for fn in (vdw.DF1, vdw.DF2):
        q0, dn, ds = vdw.q0_of(n, s, fn)
        hn = 1e-6 * n
        hs = 1e-3 * s
        qp, _, _ = vdw.q0_of(n + hn, s, fn)
        qm, _, _ = vdw.q0_of(n - hn, s, fn)
        assert np.allclose(dn, (qp - qm) / (2 * hn), rtol=1e-6, atol=1e-9)
        qp, _, _ = vdw.q0_of(n, s + hs, fn)
        qm, _, _ = vdw.q0_of(n, s - hs, fn)
        # compare the change of q0, not the slope (the gradient term can be tiny)
        assert np.allclose(ds * hs, 0.5 * (qp - qm), rtol=1e-5, atol=1e-13 * np.max(q0))


def test_q0_functionals_differ_only_through_gradient():
    n = np.array([0.01, 0.1, 1.0])
    q1, _, _ = vdw.q0_of(n, np.zeros(3), vdw.DF1)
    q2, _, _ = vdw.q0_of(n, np.zeros(3), vdw.DF2)
    assert np.array_equal(q1, q2)
    s = np.array([1e-3, 1e-2, 0.5])
    q1, _, _ = vdw.q0_of(n, s, vdw.DF1)
    q2, _, _ = vdw.q0_of(n, s, vdw.DF2)
    assert np.all(q2 > q1)     # |Z_ab| of vdW-DF2 is larger: stronger gradient term


def test_q0_range_and_cutoff():
    n = np.array([0.0, 1e-13, 1e-10, 1.0, 1e4])
    s = np.array([0.0, 0.0, 1e-10, 1e3, 0.0])
    q0, dn, ds = vdw.q0_of(n, s, vdw.DF1)
    p = vdw.Params()
    assert q0[0] == p.q_min and dn[0] == 0 and ds[0] == 0
    assert q0[1] == p.q_min and dn[1] == 0
    assert np.all(q0 >= p.q_min) and np.all(q0 <= p.q_cut)


def test_q_mesh_shape():
    q = vdw.q_mesh()
    assert len(q) == 20 and q[0] == pytest.approx(1e-5) and q[-1] == pytest.approx(5.0)
    assert np.all(np.diff(q) > 0) and np.all(np.diff(np.diff(q)) > 0)


def test_spline_basis_kronecker_and_partition():
    q = vdw.q_mesh()
    d2 = vdw.spline_basis_d2(q)
    p, _ = vdw.spline_basis(q, q, d2)
    assert np.allclose(p, np.eye(len(q)), atol=1e-13)
    x = np.linspace(q[0], q[-1], 2001)
    p, dp = vdw.spline_basis(x, q, d2)
    assert np.allclose(p.sum(axis=0), 1.0, atol=1e-12)          # constants reproduced
    assert np.allclose((q[:, None] * p).sum(axis=0), x, atol=1e-12)   # linear reproduced
    assert np.allclose(dp.sum(axis=0), 0.0, atol=1e-10)
    assert np.allclose((q[:, None] * dp).sum(axis=0), 1.0, atol=1e-10)


def test_spline_basis_matches_scipy_natural():
    from scipy.interpolate import CubicSpline
    q = vdw.q_mesh()
    d2 = vdw.spline_basis_d2(q)
    x = np.random.default_rng(2).uniform(q[0], q[-1], 300)
    p, dp = vdw.spline_basis(x, q, d2)
    for a in range(len(q)):
        cs = CubicSpline(q, np.eye(len(q))[a], bc_type="natural")
        assert np.allclose(p[a], cs(x), atol=1e-12)
        assert np.allclose(dp[a], cs(x, 1), atol=1e-10)


def test_spline_basis_c2_at_nodes():
    q = vdw.q_mesh()
    d2 = vdw.spline_basis_d2(q)
    eps = 1e-10
    for i in range(1, len(q) - 1):
        pl, dpl = vdw.spline_basis(np.array([q[i] - eps]), q, d2)
        pr, dpr = vdw.spline_basis(np.array([q[i] + eps]), q, d2)
        assert np.allclose(pl, pr, atol=1e-7)
        assert np.allclose(dpl, dpr, atol=1e-5)
