"""Pins of the oracle's kernel phi(d1, d2), radial transform and k-table.

None of these re-types the oracle's formula: each checks a property fixed by
the mathematics of the published kernel or of the transform."""
import numpy as np
import pytest

from oracle import vdw

C_ASYM = 12.0 * (4.0 * np.pi / 9.0) ** 3     # phi -> -C / (d1^2 d2^2 (d1^2 + d2^2))


def test_W_factored_equals_expanded_form():
    # The factored W used for the quadrature equals the published expanded
    # W(a, b) wherever the expanded form is well conditioned.
    rng = np.random.default_rng(1)
    a = rng.uniform(0.3, 40.0, 200)
    b = rng.uniform(0.3, 40.0, 200)
    w1 = vdw.W_dion(a, b)
    w2 = vdw.W_dion_expanded(a, b)
    assert np.max(np.abs(w1 - w2)) < 1e-10 * max(1.0, np.max(np.abs(w2)))


def test_W_small_argument_limit():
    # W(a, b) -> 2 (1/3 + 1/3 - 3/9) = 2/3 as a, b -> 0 (series of j0 and j1/x).
    assert vdw.W_dion(np.array([1e-7]), np.array([2e-7]))[0] == pytest.approx(2.0 / 3.0, rel=1e-10)


def test_phi_symmetric():
    d1 = np.array([0.1, 0.7, 1.5, 3.0, 8.0])
    d2 = np.array([2.0, 0.3, 6.0, 3.5, 1.0])
    assert np.allclose(vdw.phi_dion(d1, d2), vdw.phi_dion(d2, d1), rtol=1e-13, atol=0)


def test_phi_large_separation_asymptote():
    # Long-range limit of the published kernel: -C / (d1^2 d2^2 (d1^2 + d2^2)),
    # C = 12 (4 pi / 9)^3.  Checked with a fine quadrature (the limit needs
    # nodes well beyond a ~ d).
    d1 = np.array([20.0, 40.0, 15.0])
    d2 = np.array([20.0, 40.0, 30.0])
    ph = vdw.phi_dion(d1, d2, na=1024, a_max=256.0)
    asym = -C_ASYM / (d1 ** 2 * d2 ** 2 * (d1 ** 2 + d2 ** 2))
    assert np.all(np.abs(ph / asym - 1.0) < 0.01), ph / asym


def _int_d2_phi(lam, na, a_max):
    """int_0^inf d^2 phi(d, lam d) dd: GL panels to d = 40, analytic tail."""
    x, w = np.polynomial.legendre.leggauss(8)
    edges = np.concatenate([np.linspace(0, 2, 41), np.linspace(2, 40, 153)[1:]])
    d, wd = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        d.append(lo + (x + 1) * (hi - lo) / 2)
        wd.append(w * (hi - lo) / 2)
    d = np.concatenate(d)
    wd = np.concatenate(wd)
    ph = vdw.phi_dion(d, lam * d, na, a_max)
    tail = -C_ASYM / (lam ** 2 * (1 + lam ** 2)) / (3 * 40.0 ** 3)
    return np.sum(wd * d * d * ph) + tail, np.sum(wd * d * d * np.abs(ph))


@pytest.mark.parametrize("lam", [1.0, 2.0])
def test_phi_integrates_to_zero(lam):
    # int d^3r phi(q r, q' r) = 0: no nonlocal correlation for a uniform gas.
    # Relative to int d^2 |phi| this holds to the quadrature's accuracy.
    val, scale = _int_d2_phi(lam, 256, 64.0)
    assert abs(val) / scale < 2e-3
    val, scale = _int_d2_phi(lam, 512, 128.0)
    assert abs(val) / scale < 5e-4


def test_phi_quadrature_converged_mid_range():
    d1 = np.array([0.5, 1.0, 2.0, 5.0, 10.0])
    d2 = np.array([0.5, 1.0, 3.0, 5.0, 10.0])
    coarse = vdw.phi_dion(d1, d2, 256, 64.0)
    fine = vdw.phi_dion(d1, d2, 1024, 256.0)
    assert np.all(np.abs(coarse / fine - 1.0) < 5e-3)
    assert np.all(np.abs(coarse[:2] / fine[:2] - 1.0) < 2e-5)
    assert np.all(np.abs(coarse[:4] / fine[:4] - 1.0) < 5e-4)


def test_radial_transform_gaussian():
    # 4 pi int r^2 exp(-r^2/2) j0(k r) dr = (2 pi)^{3/2} exp(-k^2/2)
    p = vdw.Params()
    r = np.arange(p.n_r + 1) * p.dr
    k = vdw.k_grid(p)[:200]
    got = vdw.radial_transform(np.exp(-0.5 * r * r)[None, :], r, k, p.dr)[0]
    want = (2 * np.pi) ** 1.5 * np.exp(-0.5 * k * k)
    assert np.max(np.abs(got - want)) < 1e-9


def test_radial_transform_exponential():
    # 4 pi int r^2 exp(-r) j0(k r) dr = 8 pi / (1 + k^2)^2
    p = vdw.Params()
    r = np.arange(p.n_r + 1) * p.dr
    k = vdw.k_grid(p)[:100]
    got = vdw.radial_transform(np.exp(-r)[None, :], r, k, p.dr)[0]
    want = 8 * np.pi / (1 + k * k) ** 2
    assert np.max(np.abs(got - want)) < 2e-5 * 8 * np.pi


def test_radial_table_entries_are_phi(oracle_default):
    p = vdw.Params()
    _, phir = vdw.kernel_table(p)
    q = vdw.q_mesh(p)
    pairs = vdw.pair_list(p.M)
    for (a, b), i in [((3, 7), 5), ((10, 10), 100), ((0, 19), 1000), ((19, 19), 37)]:
        r = i * p.dr
        want = vdw.phi_dion(q[a] * r, q[b] * r, p.na, p.a_max)
        assert phir[pairs.index((a, b)), i] == pytest.approx(float(want), rel=1e-12, abs=1e-300)


def test_k_table_diagonal_near_zero_at_k0(oracle_default):
    # phi_aa(k = 0) = int phi d^3r ~ 0 for mesh points whose kernel has decayed
    # within r_max (q r_max >> 1); the residual is the radial discretisation.
    p = vdw.Params()
    phik = oracle_default.phik
    q = vdw.q_mesh(p)
    pairs = vdw.pair_list(p.M)
    for a in range(p.M):
        if q[a] * p.r_max < 40 or q[a] > 2.5:
            continue
        row = phik[pairs.index((a, a))]
        assert abs(row[0]) < 5e-3 * np.max(np.abs(row)), a


def test_k_table_decays(oracle_default):
    # The kernel is smooth on the scale 1/q, so phi_ab(k) has decayed by the
    # end of the table for every pair whose kernel fits in r_max.
    p = vdw.Params()
    q = vdw.q_mesh(p)
    phik = oracle_default.phik
    for i, (a, b) in enumerate(vdw.pair_list(p.M)):
        if min(q[a], q[b]) < 0.15:
            continue
        assert abs(phik[i, -1]) < 1e-3 * np.max(np.abs(phik[i])), (a, b)


def test_k_spline_matches_scipy_natural_spline(oracle_default):
    from scipy.interpolate import CubicSpline
    p = vdw.Params()
    phik = oracle_default.phik
    kg = vdw.k_grid(p)
    rng = np.random.default_rng(3)
    kq = rng.uniform(0, kg[-1] * 0.999, 500)
    got = vdw.kernel_at(kq, phik, p)
    for idx in [0, 17, 100, 209]:
        cs = CubicSpline(kg, phik[idx], bc_type="natural")
        assert np.allclose(got[idx], cs(kq), rtol=1e-10, atol=1e-12 * np.max(np.abs(phik[idx])))


def test_kernel_beyond_table_is_zero(oracle_default):
    p = vdw.Params()
    kq = np.array([(p.n_k - 1) * p.dk, p.n_k * p.dk * 1.5])
    assert np.all(vdw.kernel_at(kq, oracle_default.phik, p) == 0.0)
