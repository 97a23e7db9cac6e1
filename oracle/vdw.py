"""Oracle for the vdW-DF nonlocal correlation (Roman-Perez--Soler FFT method).

TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 numpy code written from the
paper (arXiv:1703.06999) and the kernel it cites.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU baseline of ``bench.py`` may import
or call it.  It shares no code, header, table or constant generator with the
CUDA library, and it never reads a value produced by the CUDA library.

Where each function comes from:

* ``q_mesh``            the M = 20 point q-mesh (Sec. 2, "helper splines"; the
                        mesh values are not printed, a documented log-type
                        mesh is used).
* ``spline_basis_d2`` / ``spline_basis``
                        the helper splines p_alpha(q) with p_alpha(q_beta) =
                        delta_{alpha beta}, continuous to second order
                        (Sec. 2, the equation defining a^c_{alpha beta}).
* ``q0_of``             q0(n, sigma) with PW92 correlation and the saturation
                        function h_a (Appendix, q0; saturation equation).
* ``phi_dion``          the vdW kernel phi(d1, d2) (cited at Eq. 2; published
                        form of Dion et al. 2004, double quadrature).
* ``kernel_table``      phi_{alpha beta}(k) on a discrete k-grid (Sec. 2 end,
                        "20 x 20 radial functions phi_{alpha beta}(k)").
* ``kernel_at``         interpolation of the table in k (Sec. 3 procedure,
                        step 3a; linear per the paper, natural cubic spline as
                        the default reading).
* ``energy_potential``  theta (Eq. theta), E via Eq. (enlk), F_alpha,
                        dE/dn (Eq. dedn) and dE/dsigma (Eq. dedsigma).

Readings where the paper is silent, garbled or ambiguous are stated next to
the code they affect.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
from dataclasses import dataclass, asdict

import numpy as np
from scipy.linalg import solve_banded
from scipy.special import spherical_jn

from . import build as _build

# ---------------------------------------------------------------------------
# Constants printed in the appendix (q0).
# ---------------------------------------------------------------------------
PW92_A = 0.031091
PW92_ALPHA1 = 0.2137
PW92_BETA = (7.5957, 3.5876, 1.6382, 0.49294)
Z_AB = {1: -0.8491, 2: -1.887}           # vdW-DF1, vdW-DF2
SATURATION_TERMS = 12                      # sum m = 1..12 in h_a(x)
GAMMA_DION = 4.0 * np.pi / 9.0             # gamma in h(y) = 1 - exp(-gamma y^2)

DF1 = 1
DF2 = 2


@dataclass(frozen=True)
class Params:
    """Discretisation of the method (defaults of this project).

    M, q_cut: the paper (M = 20, grid ends at 5 a.u.).  q_min, lam: mesh
    reading (log-type mesh, first point 1e-5).  n_r, r_max, n_k: radial
    table with 1024 points out to 100 bohr, k spacing 2 pi / r_max.
    na, a_max: quadrature for phi(d1, d2).  n_min: low-density cut-off.
    interp: "cubic" (natural spline in k) or "linear" (the paper's choice).
    """
    M: int = 20
    q_min: float = 1e-5
    q_cut: float = 5.0
    lam: float = 1.17
    n_r: int = 1024
    r_max: float = 100.0
    n_k: int = 1024
    na: int = 256
    a_max: float = 64.0
    n_min: float = 1e-12
    interp: str = "cubic"

    @property
    def dk(self) -> float:
        return 2.0 * np.pi / self.r_max

    @property
    def dr(self) -> float:
        return self.r_max / self.n_r


# ---------------------------------------------------------------------------
# q-mesh and helper splines p_alpha (Sec. 2).
# ---------------------------------------------------------------------------
def q_mesh(p: Params = Params()) -> np.ndarray:
    """q_alpha = q_min + (q_cut - q_min) (lam^alpha - 1) / (lam^(M-1) - 1)."""
    a = np.arange(p.M, dtype=np.float64)
    return p.q_min + (p.q_cut - p.q_min) * (p.lam ** a - 1.0) / (p.lam ** (p.M - 1) - 1.0)


def spline_basis_d2(q: np.ndarray) -> np.ndarray:
    """Second derivatives y''[alpha, i] of the natural cubic splines through
    y_alpha(q_i) = delta_{alpha i}.  Natural end conditions (y'' = 0 at both
    ends) are this project's reading: the paper only asks for continuity up
    to second order."""
    M = len(q)
    h = np.diff(q)
    A = np.zeros((M - 2, M - 2))
    for i in range(1, M - 1):
        r = i - 1
        A[r, r] = 2.0 * (h[i - 1] + h[i])
        if r > 0:
            A[r, r - 1] = h[i - 1]
        if r < M - 3:
            A[r, r + 1] = h[i]
    Y = np.eye(M)                       # column alpha: data of p_alpha
    rhs = np.zeros((M - 2, M))
    for i in range(1, M - 1):
        rhs[i - 1] = 6.0 * ((Y[i + 1] - Y[i]) / h[i] - (Y[i] - Y[i - 1]) / h[i - 1])
    inner = np.linalg.solve(A, rhs)     # (M-2) x M
    d2 = np.zeros((M, M))
    d2[:, 1:M - 1] = inner.T            # d2[alpha, i]
    return d2


def spline_interval(q: np.ndarray, mesh: np.ndarray) -> np.ndarray:
    j = np.searchsorted(mesh, q, side="right") - 1
    return np.clip(j, 0, len(mesh) - 2)


def spline_basis(qv: np.ndarray, mesh: np.ndarray, d2: np.ndarray):
    """p_alpha(q) and dp_alpha/dq for all alpha: arrays of shape (M,) + q.shape."""
    qv = np.asarray(qv, dtype=np.float64)
    M = len(mesh)
    j = spline_interval(qv, mesh)
    h = mesh[j + 1] - mesh[j]
    A = (mesh[j + 1] - qv) / h
    B = 1.0 - A
    p = np.zeros((M,) + qv.shape)
    dp = np.zeros((M,) + qv.shape)
    for alpha in range(M):
        yj = (j == alpha).astype(np.float64)
        yj1 = (j + 1 == alpha).astype(np.float64)
        d2j = d2[alpha, j]
        d2j1 = d2[alpha, j + 1]
        p[alpha] = A * yj + B * yj1 + ((A ** 3 - A) * d2j + (B ** 3 - B) * d2j1) * h * h / 6.0
        dp[alpha] = (yj1 - yj) / h + (-(3.0 * A * A - 1.0) * d2j + (3.0 * B * B - 1.0) * d2j1) * h / 6.0
    return p, dp


# ---------------------------------------------------------------------------
# q0(n, sigma) (appendix).
# ---------------------------------------------------------------------------
def pw92_eps_c(rs):
    """PW92 correlation energy per particle (Hartree) and d eps_c / d r_s,
    with the constants printed in the appendix."""
    b1, b2, b3, b4 = PW92_BETA
    srs = np.sqrt(rs)
    D = 2.0 * PW92_A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs)
    dD = 2.0 * PW92_A * (0.5 * b1 / srs + b2 + 1.5 * b3 * srs + 2.0 * b4 * rs)
    L = np.log1p(1.0 / D)
    eps = -2.0 * PW92_A * (1.0 + PW92_ALPHA1 * rs) * L
    deps = (-2.0 * PW92_A * PW92_ALPHA1 * L
            + 2.0 * PW92_A * (1.0 + PW92_ALPHA1 * rs) * dD / (D * D + D))
    return eps, deps


def saturate(x, a):
    """h_a(x) = a [1 - exp(-sum_{m=1}^{12} (x/a)^m / m)] and dh_a/dx."""
    s = np.zeros_like(x)
    ds = np.zeros_like(x)
    t = x / a
    for m in range(1, SATURATION_TERMS + 1):
        s = s + t ** m / m
        ds = ds + t ** (m - 1)
    e = np.exp(-s)
    return a * (1.0 - e), e * ds


def q0_of(n, sigma, functional: int, p: Params = Params()):
    """q0, dq0/dn and dq0/dsigma (appendix).

    Readings: the printed r_s relation is garbled; (4 pi / 3) r_s^3 n = 1 is
    used.  sigma < 0 is treated as 0.  Points with n <= n_min are returned
    with q0 = q_min and zero derivatives (the caller zeroes theta there).
    q0 below q_min is clamped to q_min with zero derivatives."""
    Z = Z_AB[functional]
    n = np.asarray(n, dtype=np.float64)
    sigma = np.maximum(np.asarray(sigma, dtype=np.float64), 0.0)
    live = n > p.n_min
    nn = np.where(live, n, 1.0)
    kF = np.cbrt(3.0 * np.pi ** 2 * nn)
    rs = np.cbrt(3.0 / (4.0 * np.pi * nn))
    eps, deps = pw92_eps_c(rs)
    G = -(Z / 36.0) * sigma / (kF * nn * nn)
    q_raw = kF - (4.0 * np.pi / 3.0) * eps + G
    dq_dn = kF / (3.0 * nn) - (4.0 * np.pi / 3.0) * deps * (-rs / (3.0 * nn)) - (7.0 / 3.0) * G / nn
    dq_ds = -(Z / 36.0) / (kF * nn * nn)
    q0, dh = saturate(q_raw, p.q_cut)
    dq0_dn = dh * dq_dn
    dq0_ds = dh * dq_ds
    low = (q0 < p.q_min) | ~live
    q0 = np.where(low, p.q_min, q0)
    dq0_dn = np.where(low, 0.0, dq0_dn)
    dq0_ds = np.where(low, 0.0, dq0_ds)
    return q0, dq0_dn, dq0_ds


# ---------------------------------------------------------------------------
# Kernel phi(d1, d2) and its tables.
# ---------------------------------------------------------------------------
_lib = None


def _clib():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_phi_batch.argtypes = [
            ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_phi_batch.restype = None
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def oracle_threads() -> int:
    return int(_clib().oracle_num_threads())


def j0(x):
    """Spherical Bessel j0(x) = sin(x)/x."""
    return np.sinc(np.asarray(x) / np.pi)


def f_j1_over_x(x):
    """f(x) = (sin x - x cos x) / x^3 = j1(x) / x; f(0) = 1/3."""
    x = np.asarray(x, dtype=np.float64)
    safe = np.where(x == 0.0, 1.0, x)
    return np.where(x == 0.0, 1.0 / 3.0, spherical_jn(1, safe) / safe)


def W_dion(a, b):
    """W(a, b) of the published kernel, written as
    2 [j0(a) f(b) + j0(b) f(a) - 3 f(a) f(b)], f(x) = (sin x - x cos x)/x^3.
    This equals 2 [(3 - a^2) b cos b sin a + (3 - b^2) a cos a sin b
    + (a^2 + b^2 - 3) sin a sin b - 3 a b cos a cos b] / (a^3 b^3) exactly
    (expand sin x - x cos x), without the cancellation at small a, b."""
    return 2.0 * (j0(a) * f_j1_over_x(b) + j0(b) * f_j1_over_x(a)
                  - 3.0 * f_j1_over_x(a) * f_j1_over_x(b))


def W_dion_expanded(a, b):
    """W(a, b) in the published expanded form (used only by a pin test)."""
    sa, ca, sb, cb = np.sin(a), np.cos(a), np.sin(b), np.cos(b)
    num = ((3.0 - a * a) * b * cb * sa + (3.0 - b * b) * a * ca * sb
           + (a * a + b * b - 3.0) * sa * sb - 3.0 * a * b * ca * cb)
    return 2.0 * num / (a ** 3 * b ** 3)


def quadrature(na: int, a_max: float):
    """Nodes a_i and weights w_i on (0, a_max): a = tan(t), t Gauss-Legendre
    on [0, atan(a_max)], w_i includes da/dt = 1 + a^2."""
    x, w = np.polynomial.legendre.leggauss(na)
    T = np.arctan(a_max)
    t = 0.5 * (x + 1.0) * T
    wt = 0.5 * T * w
    a = np.tan(t)
    return a, wt * (1.0 + a * a)


def phi_weight_matrix(na: int, a_max: float):
    a, w = quadrature(na, a_max)
    A, B = np.meshgrid(a, a, indexing="ij")
    K = (2.0 / np.pi ** 2) * np.outer(w * a * a, w * a * a) * W_dion(A, B)
    return a, np.ascontiguousarray(K)


def phi_dion(d1, d2, na: int = 256, a_max: float = 64.0) -> np.ndarray:
    """phi(d1, d2) for arrays of (d1, d2) (double quadrature in C)."""
    d1, d2 = np.broadcast_arrays(np.asarray(d1, np.float64), np.asarray(d2, np.float64))
    shape = d1.shape
    d1 = np.ascontiguousarray(d1).ravel()
    d2 = np.ascontiguousarray(d2).ravel()
    a, K = phi_weight_matrix(na, a_max)
    out = np.empty(d1.size)
    _clib().oracle_phi_batch(d1.size, d1.ctypes.data, d2.ctypes.data, na,
                             a.ctypes.data, K.ctypes.data, out.ctypes.data)
    return out.reshape(shape)


def pair_list(M: int):
    """Symmetric pairs (alpha <= beta), row-major."""
    return [(a, b) for a in range(M) for b in range(a, M)]


def radial_table(p: Params = Params()) -> np.ndarray:
    """phi_{alpha beta}(r_i) = phi(q_alpha r_i, q_beta r_i), r_i = i dr,
    i = 0..n_r; shape (n_pairs, n_r + 1)."""
    q = q_mesh(p)
    r = np.arange(p.n_r + 1) * p.dr
    pairs = pair_list(p.M)
    d1 = np.array([q[a] * r for a, _ in pairs])
    d2 = np.array([q[b] * r for _, b in pairs])
    return phi_dion(d1, d2, p.na, p.a_max)


def simpson_weights(n_intervals: int, h: float) -> np.ndarray:
    w = np.ones(n_intervals + 1)
    w[1:-1:2] = 4.0
    w[2:-1:2] = 2.0
    return w * h / 3.0


def radial_transform(f_r: np.ndarray, r: np.ndarray, k: np.ndarray, h: float) -> np.ndarray:
    """F(k) = 4 pi int_0^{r_max} r^2 f(r) j0(k r) dr, composite Simpson in r."""
    w = simpson_weights(len(r) - 1, h)
    J = j0(np.outer(r, k))                     # (n_r + 1, n_k)
    return 4.0 * np.pi * (f_r * (w * r * r)) @ J


def k_grid(p: Params = Params()) -> np.ndarray:
    return np.arange(p.n_k) * p.dk


def _cache_path(p: Params) -> str:
    key = hashlib.sha1(repr(sorted(asdict(p).items())).encode()).hexdigest()[:16]
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_cache")
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, "ktable_%s.npz" % key)


def kernel_table(p: Params = Params(), use_cache: bool = True):
    """phi_{alpha beta}(k_j), j = 0..n_k-1 for the symmetric pairs, shape
    (n_pairs, n_k); and the radial table it came from."""
    path = _cache_path(p)
    if use_cache and os.path.exists(path):
        z = np.load(path)
        return z["phik"], z["phir"]
    phir = radial_table(p)
    r = np.arange(p.n_r + 1) * p.dr
    phik = radial_transform(phir, r, k_grid(p), p.dr)
    if use_cache:
        tmp = path + ".tmp.%d.npz" % os.getpid()
        np.savez(tmp, phik=phik, phir=phir)
        os.replace(tmp, path)
    return phik, phir


def natural_spline_d2_uniform(y: np.ndarray, h: float) -> np.ndarray:
    """Second derivatives of natural cubic splines through rows of y sampled
    at uniform spacing h (y: (..., n))."""
    n = y.shape[-1]
    ab = np.zeros((3, n - 2))
    ab[0, 1:] = h
    ab[1, :] = 4.0 * h
    ab[2, :-1] = h
    rhs = 6.0 * (y[..., 2:] - 2.0 * y[..., 1:-1] + y[..., :-2]) / h
    inner = solve_banded((1, 1), ab, rhs.T).T
    d2 = np.zeros_like(y)
    d2[..., 1:-1] = inner
    return d2


def kernel_at(kabs: np.ndarray, phik: np.ndarray, p: Params = Params(), d2k=None) -> np.ndarray:
    """phi_{pair}(|k|) by interpolation in k: shape (n_pairs,) + kabs.shape.
    phi = 0 for |k| >= k_{n_k - 1} (beyond the table)."""
    kabs = np.asarray(kabs, dtype=np.float64)
    x = kabs / p.dk
    j = np.floor(x).astype(np.int64)
    inside = j < p.n_k - 1
    jj = np.where(inside, j, 0)
    B = np.where(inside, x - jj, 0.0)
    A = 1.0 - B
    yj = phik[:, jj]
    yj1 = phik[:, jj + 1]
    val = A * yj + B * yj1
    if p.interp == "cubic":
        if d2k is None:
            d2k = natural_spline_d2_uniform(phik, p.dk)
        val = val + ((A ** 3 - A) * d2k[:, jj] + (B ** 3 - B) * d2k[:, jj + 1]) * p.dk * p.dk / 6.0
    elif p.interp != "linear":
        raise ValueError(p.interp)
    return np.where(inside, val, 0.0)


# ---------------------------------------------------------------------------
# The RPS evaluation (Sec. 2 equations, Sec. 3 procedure).
# ---------------------------------------------------------------------------
def cell_volume(cell) -> float:
    return abs(float(np.linalg.det(np.asarray(cell, dtype=np.float64))))


def kabs_grid(shape, cell) -> np.ndarray:
    """|k| on the full FFT grid.  Rows of ``cell`` are the lattice vectors
    a_i; reciprocal vectors b_j with a_i . b_j = 2 pi delta_ij; indices
    m >= N/2 fold to m - N (numpy.fft.fftfreq convention).

    Reading for the Nyquist index of an even axis (m = -N/2, whose sign is
    ambiguous): it enters |k|^2 = sum_ij g_ij m_i m_j (g = B B^T) through
    the diagonal term only; its cross terms, whose sign would flip between
    +N/2 and -N/2, are dropped.  |k(m)| = |k(-m)| then holds on the whole
    grid, so F_alpha(r) stays real.  For orthogonal cells this is the plain
    |k|."""
    cell = np.asarray(cell, dtype=np.float64)
    Bm = 2.0 * np.pi * np.linalg.inv(cell).T          # rows b_j
    g = Bm @ Bm.T
    m = [np.fft.fftfreq(s, 1.0 / s) for s in shape]
    c = [np.where((s % 2 == 0) & (mi == -(s // 2)), 0.0, mi) for s, mi in zip(shape, m)]
    M = np.meshgrid(*m, indexing="ij")
    Cm = np.meshgrid(*c, indexing="ij")
    k2 = sum(g[i, i] * M[i] * M[i] for i in range(3))
    for i in range(3):
        for j in range(i + 1, 3):
            k2 = k2 + 2.0 * g[i, j] * Cm[i] * Cm[j]
    return np.sqrt(k2)


@dataclass
class Result:
    energy: float
    dedn: np.ndarray
    dedsigma: np.ndarray
    q0: np.ndarray = None
    theta: np.ndarray = None
    F: np.ndarray = None


class Oracle:
    """FP64 oracle holding the mesh, spline basis and kernel table."""

    def __init__(self, p: Params = Params(), phik=None):
        self.p = p
        self.mesh = q_mesh(p)
        self.d2q = spline_basis_d2(self.mesh)
        if phik is None:
            phik, _ = kernel_table(p)
        self.phik = phik
        self.d2k = natural_spline_d2_uniform(phik, p.dk) if p.interp == "cubic" else None
        self.pairs = pair_list(p.M)

    def theta(self, n, sigma, functional):
        """theta_alpha(r) = n(r) p_alpha(q0(r)); zero where n <= n_min."""
        q0, dq_dn, dq_ds = q0_of(n, sigma, functional, self.p)
        pa, dpa = spline_basis(q0, self.mesh, self.d2q)
        live = np.asarray(n) > self.p.n_min
        theta = np.where(live, n * pa, 0.0)
        return theta, q0, dq_dn, dq_ds, pa, dpa, live

    def kernel_matrix(self, kabs):
        """Full symmetric M x M kernel at the given |k| values: (M, M, K)."""
        vals = kernel_at(kabs, self.phik, self.p, self.d2k)
        M = self.p.M
        phi = np.empty((M, M) + kabs.shape)
        for idx, (a, b) in enumerate(self.pairs):
            phi[a, b] = vals[idx]
            phi[b, a] = vals[idx]
        return phi

    def energy_potential(self, n, sigma, cell, functional, keep=False,
                         chunk: int = 32768) -> Result:
        n = np.asarray(n, dtype=np.float64)
        sigma = np.asarray(sigma, dtype=np.float64)
        shape = n.shape
        N = n.size
        omega = cell_volume(cell)
        theta, q0, dq_dn, dq_ds, pa, dpa, live = self.theta(n, sigma, functional)
        M = self.p.M
        # theta_alpha(k): unnormalised forward DFT of each field (full grid).
        th_k = np.fft.fftn(theta, axes=(1, 2, 3)).reshape(M, N)
        kabs = kabs_grid(shape, cell).reshape(N)
        F_k = np.empty_like(th_k)
        esum = 0.0
        for s in range(0, N, chunk):
            e = min(N, s + chunk)
            phi = self.kernel_matrix(kabs[s:e])                # (M, M, c)
            Fk = np.einsum("abk,bk->ak", phi, th_k[:, s:e])    # F_alpha(k)
            F_k[:, s:e] = Fk
            esum += float(np.sum(np.real(np.conj(th_k[:, s:e]) * Fk)))
        energy = 0.5 * omega / (N * float(N)) * esum
        # F_alpha(r) = (1/N) sum_k F_alpha(k) e^{i k r}
        F = np.real(np.fft.ifftn(F_k.reshape((M,) + shape), axes=(1, 2, 3)))
        dedn = np.sum(F * (pa + n * dpa * dq_dn), axis=0)
        dedsigma = n * np.sum(F * dpa, axis=0) * dq_ds
        dedn = np.where(live, dedn, 0.0)
        dedsigma = np.where(live, dedsigma, 0.0)
        res = Result(energy, dedn, dedsigma)
        if keep:
            res.q0, res.theta, res.F = q0, theta, F
        return res


def calculate(n, sigma, cell, functional=DF1, p: Params = Params()):
    """Convenience: (E, dE/dn, dE/dsigma) in FP64."""
    r = Oracle(p).energy_potential(n, sigma, cell, functional)
    return r.energy, r.dedn, r.dedsigma
