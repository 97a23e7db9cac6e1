"""Pins of the oracle's energy and potential (Eq. enlk, Eq. dedn, Eq. dedsigma)."""
import numpy as np
import pytest

from oracle import vdw
from paper_1703_06999_gb300 import inputs


def _small(seed=0, shape=(12, 10, 9), L=(7.0, 6.0, 6.5), natoms=3, cell=None):
    if cell is None:
        cell = np.diag(L)
    g = np.random.default_rng(seed)
    atoms = [(float(g.uniform(1, 4)), float(g.uniform(0.8, 1.6)),
              tuple(g.uniform(0, 1, 3) @ cell)) for _ in range(natoms)]
    s = inputs.make_system(shape, cell, atoms, 1, 1e-6)
    return s.n.numpy(), s.sigma.numpy(), cell


def test_uniform_density_closed_form(oracle_default):
    # Only k = 0 survives: E = 1/2 Omega n^2 p^T phi(0) p.
    o = oracle_default
    cell = np.diag([5.0, 6.0, 7.0])
    n0 = 0.02
    n = np.full((6, 5, 4), n0)
    res = o.energy_potential(n, np.zeros_like(n), cell, vdw.DF1)
    q0, dq, _ = vdw.q0_of(np.array([n0]), np.zeros(1), vdw.DF1)
    p, dp = vdw.spline_basis(q0, o.mesh, o.d2q)
    phi0 = o.kernel_matrix(np.zeros(1))[:, :, 0]
    omega = 210.0
    want = 0.5 * omega * n0 ** 2 * float(p[:, 0] @ phi0 @ p[:, 0])
    assert res.energy == pytest.approx(want, rel=1e-12)
    # dE/dn is uniform and equals d/dn [E_uniform(n)] / Omega
    assert np.ptp(res.dedn) < 1e-12 * abs(res.dedn.mean())
    h = 1e-6 * n0
    ep = o.energy_potential(n + h, np.zeros_like(n), cell, vdw.DF1).energy
    em = o.energy_potential(n - h, np.zeros_like(n), cell, vdw.DF1).energy
    assert res.dedn.mean() == pytest.approx((ep - em) / (2 * h) / omega, rel=1e-6)


def _brute_band_limited(o, n, sigma, cell, functional):
    """E = 1/2 dV^2 sum_ij sum_ab theta_a(r_i) Phi_ab(r_i - r_j) theta_b(r_j),
    Phi_ab(R) = (1/Omega) sum_{k on the grid} phi_ab(|k|) e^{i k.R}, by
    explicit sums (no FFT)."""
    shape = n.shape
    N = n.size
    omega = vdw.cell_volume(cell)
    theta = o.theta(n, sigma, functional)[0].reshape(o.p.M, N)
    kabs = vdw.kabs_grid(shape, cell).reshape(N)
    phi = o.kernel_matrix(kabs)                               # (M, M, N)
    idx = np.stack(np.meshgrid(*[np.arange(s) for s in shape], indexing="ij"), -1).reshape(N, 3)
    m = np.stack(np.meshgrid(*[np.fft.fftfreq(s, 1.0 / s) for s in shape], indexing="ij"), -1).reshape(N, 3)
    # Phi for every displacement d = i - j (mod grid), indexed like the grid
    phase = np.exp(2j * np.pi * (idx / np.array(shape)) @ m.T)   # (disp, k)
    Phi = np.real(np.einsum("abk,dk->abd", phi, phase)) / omega  # (M, M, disp)
    dV = omega / N
    E = 0.0
    for i in range(N):
        d = (idx[i] - idx) % np.array(shape)
        didx = (d[:, 0] * shape[1] + d[:, 1]) * shape[2] + d[:, 2]
        E += np.einsum("a,abj,bj->", theta[:, i], Phi[:, :, didx], theta)
    return 0.5 * dV * dV * E


@pytest.mark.parametrize("shape,cell", [
    ((6, 4, 5), np.diag([4.0, 3.5, 4.5])),
    ((5, 5, 3), np.array([[4.0, 0.0, 0.0], [1.2, 3.8, 0.0], [0.4, -0.7, 3.0]])),
    ((4, 6, 4), np.array([[4.0, 0.3, 0.0], [0.9, 3.8, 0.0], [0.4, -0.7, 3.3]])),
])
def test_fft_energy_equals_real_space_double_sum(oracle_default, shape, cell):
    n, s, cell = _small(1, shape, cell=cell)
    e_fft = oracle_default.energy_potential(n, s, cell, vdw.DF1).energy
    e_bru = _brute_band_limited(oracle_default, n, s, cell, vdw.DF1)
    assert e_fft == pytest.approx(e_bru, rel=1e-11)


def test_F_is_real_for_triclinic_even_grid(oracle_default):
    cell = np.array([[4.0, 0.3, 0.0], [0.9, 3.8, 0.0], [0.4, -0.7, 3.3]])
    n, s, cell = _small(2, (4, 6, 4), cell=cell)
    o = oracle_default
    theta = o.theta(n, s, vdw.DF1)[0]
    thk = np.fft.fftn(theta, axes=(1, 2, 3))
    kabs = vdw.kabs_grid(n.shape, cell)
    Fk = np.einsum("abxyz,bxyz->axyz", o.kernel_matrix(kabs), thk)
    F = np.fft.ifftn(Fk, axes=(1, 2, 3))
    assert np.max(np.abs(F.imag)) < 1e-13 * np.max(np.abs(F.real))


@pytest.mark.parametrize("interp", ["cubic", "linear"])
def test_potential_matches_finite_differences(oracle_default, oracle_linear, interp):
    o = oracle_default if interp == "cubic" else oracle_linear
    n, s, cell = _small(3)
    res = o.energy_potential(n, s, cell, vdw.DF1)
    dV = vdw.cell_volume(cell) / n.size
    rng = np.random.default_rng(7)
    pts = [tuple(rng.integers(0, d) for d in n.shape) for _ in range(4)]
    pts.append(tuple(np.unravel_index(np.argmax(n), n.shape)))
    for pt in pts:
        h = 1e-4 * n[pt]
        nn = n.copy(); nn[pt] += h
        ep = o.energy_potential(nn, s, cell, vdw.DF1).energy
        nn[pt] -= 2 * h
        em = o.energy_potential(nn, s, cell, vdw.DF1).energy
        fd = (ep - em) / (2 * h) / dV
        assert res.dedn[pt] == pytest.approx(fd, rel=2e-6, abs=1e-9 * np.max(np.abs(res.dedn)))
        hs = 1e-4 * max(s[pt], 1e-8)
        ss = s.copy(); ss[pt] += hs
        ep = o.energy_potential(n, ss, cell, vdw.DF1).energy
        ss[pt] -= 2 * hs
        em = o.energy_potential(n, ss, cell, vdw.DF1).energy
        fd = (ep - em) / (2 * hs) / dV
        assert res.dedsigma[pt] == pytest.approx(fd, rel=2e-6, abs=1e-9 * np.max(np.abs(res.dedsigma)))


def test_translation_by_grid_points(oracle_default):
    n, s, cell = _small(4)
    r0 = oracle_default.energy_potential(n, s, cell, vdw.DF2)
    sh = (3, -2, 5)
    r1 = oracle_default.energy_potential(np.roll(n, sh, (0, 1, 2)), np.roll(s, sh, (0, 1, 2)), cell, vdw.DF2)
    assert r1.energy == pytest.approx(r0.energy, rel=1e-12)
    assert np.allclose(r1.dedn, np.roll(r0.dedn, sh, (0, 1, 2)), rtol=1e-10, atol=1e-14)
    assert np.allclose(r1.dedsigma, np.roll(r0.dedsigma, sh, (0, 1, 2)), rtol=1e-10, atol=1e-14)


def test_supercell_extensive(oracle_default):
    n, s, cell = _small(5)
    r0 = oracle_default.energy_potential(n, s, cell, vdw.DF1)
    cell2 = cell.copy(); cell2[0] *= 2
    r2 = oracle_default.energy_potential(np.tile(n, (2, 1, 1)), np.tile(s, (2, 1, 1)), cell2, vdw.DF1)
    assert r2.energy == pytest.approx(2 * r0.energy, rel=1e-11)
    assert np.allclose(r2.dedn, np.tile(r0.dedn, (2, 1, 1)), rtol=1e-9, atol=1e-13)


def test_df1_equals_df2_without_gradient(oracle_default):
    n, s, cell = _small(6)
    z = np.zeros_like(s)
    e1 = oracle_default.energy_potential(n, z, cell, vdw.DF1)
    e2 = oracle_default.energy_potential(n, z, cell, vdw.DF2)
    assert e1.energy == e2.energy
    assert np.array_equal(e1.dedn, e2.dedn)
    e1 = oracle_default.energy_potential(n, s, cell, vdw.DF1).energy
    e2 = oracle_default.energy_potential(n, s, cell, vdw.DF2).energy
    assert e1 != e2


def test_hello_example_finite_and_deterministic(oracle_default):
    h = inputs.hello_example()
    a = oracle_default.energy_potential(h.n.numpy(), h.sigma.numpy(), h.cell, vdw.DF1)
    b = oracle_default.energy_potential(h.n.numpy(), h.sigma.numpy(), h.cell, vdw.DF1)
    assert np.isfinite(a.energy) and a.energy == b.energy
    assert np.all(np.isfinite(a.dedn)) and np.array_equal(a.dedn, b.dedn)


@pytest.mark.parametrize("cell", [
    np.diag([4.2, 3.6, 4.0]),
    np.array([[4.2, 0.0, 0.0], [1.1, 3.7, 0.0], [-0.6, 0.8, 3.9]]),
])
def test_gaussian_kernel_table_matches_real_space_physics(cell):
    # Replace the vdW table by phi_ab(k) = exp(-k^2/2) for every pair.  Then
    # sum_a theta_a = n (partition of unity), F_a = Phi * n for all a, and
    # E = 1/2 dV^2 sum_ij n_i n_j Phi(r_i - r_j), dE/dn = dV sum_j Phi(r_i - r_j) n_j,
    # dE/dsigma = 0, with the real-space kernel Phi(R) = (2 pi)^{-3/2}
    # sum_images exp(-|R + T|^2 / 2).  Pins |k| (2 pi, cell metric), the
    # k-interpolation and the FFT normalisation against real-space sums.
    p = vdw.Params()
    kg = vdw.k_grid(p)
    phik = np.tile(np.exp(-0.5 * kg * kg), (len(vdw.pair_list(p.M)), 1))
    o = vdw.Oracle(p, phik=phik)
    shape = (10, 9, 10)
    n, s, cell = _small(9, shape, cell=cell)
    res = o.energy_potential(n, s, cell, vdw.DF1)
    N = n.size
    dV = vdw.cell_volume(cell) / N
    frac = np.stack(np.meshgrid(*[np.arange(v) / v for v in shape], indexing="ij"), -1).reshape(N, 3)
    r = frac @ cell
    nf = n.reshape(N)
    conv = np.zeros(N)
    for i in range(-2, 3):
        for j in range(-2, 3):
            for k in range(-2, 3):
                T = i * cell[0] + j * cell[1] + k * cell[2]
                d = r[:, None, :] - r[None, :, :] + T
                conv += np.exp(-0.5 * np.sum(d * d, -1)) @ nf
    conv *= (2 * np.pi) ** -1.5 * dV
    e_real = 0.5 * dV * float(nf @ conv)
    assert res.energy == pytest.approx(e_real, rel=1e-6)
    assert np.allclose(res.dedn.reshape(N), conv, rtol=1e-5, atol=1e-7 * np.max(np.abs(conv)))
    assert np.max(np.abs(res.dedsigma)) < 1e-9 * np.max(np.abs(conv))
