"""Spin-polarised vdW-DF nonlocal correlation (svdW-DF), FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring): only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it.

The paper announces the spin-polarised form (Sec. 1 and the outlook) and
cites Thonhauser et al., PRL 115, 136402 (2015) for it without printing it.
That published definition keeps everything of the unpolarised method but
q0:

* theta_alpha = n p_alpha(q0) with the total density n = n_up + n_dn, the
  same kernel and the same energy (Eq. enlk);
* q0 = -(4 pi / 3) eps_xc^0 as in the appendix, with the exchange part
  spin-scaled, E_x[n_up, n_dn] = (E_x[2 n_up] + E_x[2 n_dn]) / 2, each spin
  channel carrying the gradient correction of its own doubled density;
* the LDA correlation is PW92 with its spin interpolation (Perdew and Wang,
  PRB 45, 13244 (1992)):
      eps_c(r_s, zeta) = eps_0 + alpha_c f(zeta) / f''(0) (1 - zeta^4)
                         + (eps_1 - eps_0) f(zeta) zeta^4,
  f(zeta) = [(1 + zeta)^(4/3) + (1 - zeta)^(4/3) - 2] / (2^(4/3) - 2),
  eps_0 with the appendix's constants, eps_1 and -alpha_c with PW92's
  ferromagnetic and spin-stiffness parameter sets.

Written out, with k_s = (6 pi^2 n_s)^(1/3) (the Fermi wave vector of the
density 2 n_s) and a_s = n_s k_s:

    q_raw = sum_s [ a_s / n - (Z_ab / 36) sigma_ss / (n a_s) ]
            - (4 pi / 3) eps_c(r_s, zeta),

the exchange of channel s being (n_s / n) k_s [1 - (Z_ab / 9) s_s^2] with
s_s^2 = |2 grad n_s|^2 / (4 k_s^2 (2 n_s)^2) = sigma_ss / (4 k_s^2 n_s^2),

so at zeta = 0 (n_s = n / 2, sigma_ss = sigma / 4) q_raw is the appendix's
k_F - (4 pi / 3) eps_c - (Z_ab / 36) sigma / (k_F n^2).

Potentials: dE/dn_s = sum_alpha F_alpha [p_alpha + n p'_alpha dq0/dn_s] and
dE/dsigma_ss = n sum_alpha F_alpha p'_alpha dq0/dsigma_ss (Eq. dedn and
Eq. dedsigma with the chain rule through q0); E does not depend on
sigma_{up,dn}.

Pins (tests/test_oracle_spin.py): the unpolarised limit equals the
appendix's q0 and the unpolarised energy and potentials; the exchange obeys
spin scaling through the unpolarised q0; PW92's A and beta1, beta2 of all
three parameter sets follow its high-density expansion; f''(0) and the
endpoints of the interpolation; finite differences of q0 and of E.
Parity unpinned: alpha1, beta3 and beta4 of the ferromagnetic and
spin-stiffness sets (PW92's fitted constants, as published; nothing outside
them fixes their values).

Readings (the paper is silent on all of them): n_s < 0 and sigma_ss < 0 are
treated as 0; the point is live when n = n_up + n_dn > n_min (as in the
unpolarised form); a spin channel with n_s <= n_min contributes no exchange
term and has zero derivatives with respect to its own n_s and sigma_ss (its
term vanishes as n_s^(4/3) while its gradient part is 0/0).
"""
from __future__ import annotations

import numpy as np

from . import vdw

# PW92 parameter sets (A, alpha1, beta1, beta2, beta3, beta4): the
# unpolarised set is the appendix's; the ferromagnetic one and the one of
# -alpha_c (spin stiffness) are PW92's.
PW92_P0 = (vdw.PW92_A, vdw.PW92_ALPHA1) + tuple(vdw.PW92_BETA)
PW92_P1 = (0.015545, 0.20548, 14.1189, 6.1977, 3.3662, 0.62517)
PW92_PA = (0.016887, 0.11125, 10.357, 3.6231, 0.88026, 0.49671)
FZ20 = 1.709921                       # f''(0)
_FDEN = 2.0 ** (4.0 / 3.0) - 2.0


def pw92_G(rs, par):
    """G(r_s) = -2A (1 + alpha1 r_s) ln[1 + 1 / (2A (b1 r_s^1/2 + b2 r_s +
    b3 r_s^3/2 + b4 r_s^2))] and dG/dr_s (PW92's one functional form)."""
    A, a1, b1, b2, b3, b4 = par
    srs = np.sqrt(rs)
    D = 2.0 * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs)
    dD = 2.0 * A * (0.5 * b1 / srs + b2 + 1.5 * b3 * srs + 2.0 * b4 * rs)
    L = np.log1p(1.0 / D)
    g = -2.0 * A * (1.0 + a1 * rs) * L
    dg = -2.0 * A * a1 * L + 2.0 * A * (1.0 + a1 * rs) * dD / (D * D + D)
    return g, dg


def f_zeta(z):
    """PW92's spin interpolation f(zeta) and f'(zeta)."""
    up, dn = np.cbrt(1.0 + z), np.cbrt(1.0 - z)
    f = ((1.0 + z) * up + (1.0 - z) * dn - 2.0) / _FDEN
    df = (4.0 / 3.0) * (up - dn) / _FDEN
    return f, df


def pw92_eps_c_spin(rs, z):
    """eps_c(r_s, zeta), d eps_c / d r_s, d eps_c / d zeta (PW92)."""
    e0, d0 = pw92_G(rs, PW92_P0)
    e1, d1 = pw92_G(rs, PW92_P1)
    ga, dga = pw92_G(rs, PW92_PA)            # ga = -alpha_c
    f, df = f_zeta(z)
    z3 = z * z * z
    z4 = z3 * z
    eps = e0 - ga * f / FZ20 * (1.0 - z4) + (e1 - e0) * f * z4
    deps_rs = d0 - dga * f / FZ20 * (1.0 - z4) + (d1 - d0) * f * z4
    deps_z = -ga / FZ20 * (df * (1.0 - z4) - 4.0 * z3 * f) + (e1 - e0) * (df * z4 + 4.0 * z3 * f)
    return eps, deps_rs, deps_z


def q_raw_spin(n_up, n_dn, s_up, s_dn, functional: int, p: vdw.Params = vdw.Params()):
    """q_raw (before saturation), its partial derivatives (d/dn_up, d/dn_dn,
    d/dsigma_upup, d/dsigma_dndn), the exchange part alone, and the live mask."""
    Z = vdw.Z_AB[functional]
    c = Z / 36.0
    nu = np.maximum(np.asarray(n_up, dtype=np.float64), 0.0)
    nd = np.maximum(np.asarray(n_dn, dtype=np.float64), 0.0)
    su = np.maximum(np.asarray(s_up, dtype=np.float64), 0.0)
    sd = np.maximum(np.asarray(s_dn, dtype=np.float64), 0.0)
    n = nu + nd
    live = n > p.n_min
    nn = np.where(live, n, 1.0)
    xs, dx_own, dx_other, dx_sig = [], [], [], []
    for ns, ss in ((nu, su), (nd, sd)):
        on = live & (ns > p.n_min)
        m = np.where(on, ns, 1.0)
        k = np.cbrt(6.0 * np.pi ** 2 * m)
        a = m * k                                       # n_s k_s, proportional to n_s^(4/3)
        x = a / nn - c * ss / (nn * a)
        own = (4.0 / 3.0) * k / nn - a / nn ** 2 + c * ss / (nn * a) * (1.0 / nn + (4.0 / 3.0) / m)
        other = -a / nn ** 2 + c * ss / (nn ** 2 * a)
        sig = -c / (nn * a)
        xs.append(np.where(on, x, 0.0))
        dx_own.append(np.where(on, own, 0.0))
        dx_other.append(np.where(on, other, 0.0))
        dx_sig.append(np.where(on, sig, 0.0))
    zeta = np.where(live, (nu - nd) / nn, 0.0)
    rs = np.cbrt(3.0 / (4.0 * np.pi * nn))
    eps, deps_rs, deps_z = pw92_eps_c_spin(rs, zeta)
    kc = 4.0 * np.pi / 3.0
    xsum = xs[0] + xs[1]
    q = xsum - kc * eps
    # d(-kc eps)/dn_s = -kc [deps/drs (-r_s / 3n) + deps/dzeta dzeta/dn_s]
    common = kc * deps_rs * rs / (3.0 * nn)
    dq_up = dx_own[0] + dx_other[1] + common - kc * deps_z * (1.0 - zeta) / nn
    dq_dn = dx_own[1] + dx_other[0] + common + kc * deps_z * (1.0 + zeta) / nn
    return q, (dq_up, dq_dn, dx_sig[0], dx_sig[1]), xsum, live


def q0_spin(n_up, n_dn, s_up, s_dn, functional: int, p: vdw.Params = vdw.Params()):
    """q0 and (dq0/dn_up, dq0/dn_dn, dq0/dsigma_upup, dq0/dsigma_dndn) with the
    appendix's saturation and clamps (q0 < q_min -> q_min, zero derivatives;
    dead points -> q_min, zero derivatives)."""
    q, dq, _, live = q_raw_spin(n_up, n_dn, s_up, s_dn, functional, p)
    q0, dh = vdw.saturate(q, p.q_cut)
    low = (q0 < p.q_min) | ~live
    q0 = np.where(low, p.q_min, q0)
    d = tuple(np.where(low, 0.0, dh * x) for x in dq)
    return q0, d, live


def energy_potential_spin(o: vdw.Oracle, n_up, n_dn, s_up, s_dn, cell, functional):
    """E, (dE/dn_up, dE/dn_dn), (dE/dsigma_upup, dE/dsigma_dndn) on the grid
    (Eq. enlk with theta of the total density; potentials by the chain rule
    through the spin q0)."""
    nu = np.asarray(n_up, dtype=np.float64)
    nd = np.asarray(n_dn, dtype=np.float64)
    n = np.maximum(nu, 0.0) + np.maximum(nd, 0.0)
    shape = n.shape
    N = n.size
    q0, dq, live = q0_spin(nu, nd, s_up, s_dn, functional, o.p)
    pa, dpa = vdw.spline_basis(q0, o.mesh, o.d2q)
    theta = np.where(live, n * pa, 0.0)
    M = o.p.M
    th_k = np.fft.fftn(theta, axes=(1, 2, 3)).reshape(M, N)
    kabs = vdw.kabs_grid(shape, cell).reshape(N)
    F_k = np.einsum("abk,bk->ak", o.kernel_matrix(kabs), th_k)
    energy = 0.5 * vdw.cell_volume(cell) / (N * float(N)) * float(np.sum(np.real(np.conj(th_k) * F_k)))
    F = np.real(np.fft.ifftn(F_k.reshape((M,) + shape), axes=(1, 2, 3)))
    S0 = np.sum(F * pa, axis=0)                 # sum_a F_a p_a
    S1 = n * np.sum(F * dpa, axis=0)            # n sum_a F_a p'_a
    dedn = tuple(np.where(live, S0 + S1 * d, 0.0) for d in dq[:2])
    deds = tuple(np.where(live, S1 * d, 0.0) for d in dq[2:])
    return energy, dedn, deds
