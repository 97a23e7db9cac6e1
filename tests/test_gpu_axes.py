"""GPU parity on the axis lengths the workloads use, on inputs at the edges
of the method's domain, and on the 192^3 ligand-shell workload.

* Every FFT length with a compiled register codelet above 64 (72, 128, 144,
  160, 192, 224, 256) is put on x, on y and on z of a thin grid, in both
  precisions.  The other two axes are short, so the oracle stays cheap.
* A density with exact zeros, negative values and values just below and
  above the low-density cut-off n_min = 1e-12, negative sigma entries and
  saturating densities, compared element by element.
* The 192^3 ligand-shell-like system (200 exponentials, vacuum near 1e-8)
  against the oracle in both precisions (slow: the oracle takes about a
  minute on one core).

Tolerances as in test_gpu_parity: FP64 energy 1e-10 relative and potential
1e-9 of its max norm; FP32-mixed |dE| <= 1e-6 Ha and potential 1e-5 of its
max norm."""
import numpy as np
import pytest

from oracle import vdw
from paper_1703_06999_gb300 import inputs

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1703_06999_gb300.binding")

TOL = {0: (1e-10, 1e-9), 1: (1e-6, 1e-5)}


def _check(res, ref, prec):
    e, dn, ds = res
    etol, ptol = TOL[prec]
    assert np.isfinite(e) and np.all(np.isfinite(dn)) and np.all(np.isfinite(ds))
    if prec == B.FP64:
        assert abs(e - ref.energy) <= etol * max(abs(ref.energy), 1e-3), (e, ref.energy)
    else:
        assert abs(e - ref.energy) <= etol, (e, ref.energy)
    assert np.max(np.abs(dn - ref.dedn)) <= ptol * max(np.max(np.abs(ref.dedn)), 1e-300)
    assert np.max(np.abs(ds - ref.dedsigma)) <= ptol * max(np.max(np.abs(ref.dedsigma)), 1e-300)


def _thin(L, axis):
    shape = [6, 8, 10]
    shape[axis] = L
    lengths = [3.0, 4.0, 4.5]
    lengths[axis] = 0.2 * L
    atoms = []
    g = np.random.default_rng(L + 7 * axis)
    for _ in range(3):
        c = g.uniform(0, 1, 3) * lengths
        atoms.append((float(g.uniform(1, 6)), float(g.uniform(1.0, 2.5)), tuple(c)))
    return inputs.make_system(tuple(shape), np.diag(lengths), atoms, 1 + axis % 2)


LENGTHS = [72, 128, 144, 160, 192, 224, 256]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("axis", [0, 1, 2], ids=["x", "y", "z"])
@pytest.mark.parametrize("L", LENGTHS)
def test_codelet_lengths_on_each_axis(oracle_default, L, axis, prec):
    s = _thin(L, axis)
    n, sg = s.n.numpy(), s.sigma.numpy()
    ref = oracle_default.energy_potential(n, sg, s.cell, s.functional)
    f = B.Functional(s.shape, s.cell, s.functional, prec)
    try:
        _check(f.calculate(n, sg), ref, prec)
    finally:
        f.close()


def _edge_system():
    """A small density pushed to the edges of the method's domain: exact
    zeros, negative values (numerical noise a host code may pass), values
    just below and just above n_min = 1e-12, a few large densities whose q0
    saturates at q_cut = 5, and negative sigma entries."""
    s = inputs.make_system((24, 20, 18), np.diag([8.0, 7.0, 6.5]),
                           [(4.0, 1.6, (2.0, 2.0, 2.0)), (2.0, 1.1, (6.0, 5.0, 4.0))], 2)
    n = s.n.numpy().copy()
    sg = s.sigma.numpy().copy()
    g = np.random.default_rng(3)
    flat_n, flat_s = n.reshape(-1), sg.reshape(-1)
    n[:, :, 12:15] = 0.0                              # an exactly empty slab
    idx = g.choice(flat_n.size, 510, replace=False)
    vals = np.concatenate([np.full(100, -1e-14), np.full(100, 1e-13), np.full(100, 1e-12),
                           np.full(100, 1.0000001e-12), np.full(100, 3e-12),
                           np.full(10, 15.0)])      # q_raw / q_cut > 1.5: q0 = q_cut to FP64 precision
    flat_n[idx] = vals
    neg = g.choice(flat_s.size, 400, replace=False)
    flat_s[neg] = -np.abs(flat_s[neg]) - 1e-9        # negative sigma: treated as 0
    return s, n, sg


@pytest.mark.parametrize("prec", [0, 1])
def test_low_density_and_saturation_edges(oracle_default, prec):
    s, n, sg = _edge_system()
    ref = oracle_default.energy_potential(n, sg, s.cell, s.functional)
    f = B.Functional(s.shape, s.cell, s.functional, prec)
    try:
        got = f.calculate(n, sg)
    finally:
        f.close()
    _check(got, ref, prec)
    dead = n <= 1e-12
    assert np.all(got[1][dead] == 0.0) and np.all(got[2][dead] == 0.0)
    # the q0 < q_min clamp cannot be reached by a live point: k_F(n_min) is
    # about 3.1e-4 > q_min = 1e-5 and the other two terms are non-negative
    q0, _, _ = vdw.q0_of(np.array([1.0000001e-12]), np.array([0.0]), 1)
    assert q0[0] > 3e-4


def test_sigma_sign_only_enters_as_zero(oracle_default):
    # sigma < 0 means sigma = 0 on both sides: replacing every negative entry
    # by 0 gives the same GPU result bit for bit
    s, n, sg = _edge_system()
    clipped = np.maximum(sg, 0.0)
    for prec in (0, 1):
        f = B.Functional(s.shape, s.cell, s.functional, prec)
        try:
            a = f.calculate(n, sg)
            b = f.calculate(n, clipped)
        finally:
            f.close()
        assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.slow
def test_ligand_shell_192_against_oracle(oracle_default):
    import torch
    s = inputs.ligand_shell(0, device=torch.device("cuda:0"))
    n, sg = s.n.cpu().numpy(), s.sigma.cpu().numpy()
    ref = oracle_default.energy_potential(n, sg, s.cell, s.functional)
    for prec in (B.FP32_MIXED, B.FP64):
        f = B.Functional(s.shape, s.cell, s.functional, prec)
        try:
            _check(f.calculate(n, sg), ref, prec)
        finally:
            f.close()


@pytest.mark.parametrize("axis", [0, 1, 2], ids=["x", "y", "z"])
def test_axis_640_fp32_and_fp64_limit(oracle_default, axis):
    # 640 points, the paper's density-grid axis (performance section): the
    # FP32-mixed form takes it on any axis (generic Stockham stages); the FP64
    # form's tiles of one 640-point pencil of 20 complex fields do not fit
    # shared memory, and it says so (EINVAL) instead of running
    s = _thin(640, axis)
    n, sg = s.n.numpy(), s.sigma.numpy()
    ref = oracle_default.energy_potential(n, sg, s.cell, s.functional)
    f = B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED)
    try:
        _check(f.calculate(n, sg), ref, B.FP32_MIXED)
    finally:
        f.close()
    with pytest.raises(B.VdwgbError) as ei:
        B.Functional(s.shape, s.cell, s.functional, B.FP64)
    assert ei.value.code == -1


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("n", [300, 448])
def test_axes_above_256_points_in_several_tensor_copies(oracle_default, n, axis):
    # x / y tiles longer than the 256 rows of one tensor copy go in several
    # copies of a divisor of the axis (300: 100 or 150 rows, 448: 224), each
    # landing at an aligned offset of the tile buffer
    s = _thin(n, axis)
    sn, sg = s.n.numpy(), s.sigma.numpy()
    ref = oracle_default.energy_potential(sn, sg, s.cell, s.functional)
    f = B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED)
    try:
        _check(f.calculate(sn, sg), ref, B.FP32_MIXED)
    finally:
        f.close()


def _shell160():
    """A ligand-shell-like density on 160^3 points in a 27.4 bohr cell (one
    quarter of the paper's (58 Angstrom)^3 box along each axis)."""
    g = np.random.default_rng(640)
    L = 109.6 / 4
    c0 = np.array([L / 2] * 3)
    atoms = []
    for _ in range(12):
        v = g.normal(size=3)
        v *= g.uniform(0, 3.0) / np.linalg.norm(v)
        atoms.append((float(g.uniform(6, 8)), float(g.uniform(2, 3)), tuple(c0 + v)))
    for _ in range(8):
        u = g.normal(size=3)
        u /= np.linalg.norm(u)
        for k in range(4):
            atoms.append((float(g.uniform(1, 6)), float(g.uniform(1, 2.5)), tuple(c0 + (4.0 + 1.2 * k) * u)))
    import torch
    dev = torch.device("cuda:0")
    return inputs.make_system((160, 160, 160), np.diag([L, L, L]), atoms, 1, device=dev)


@pytest.mark.slow
def test_grid_640_cubed_supercell_of_160_cubed():
    # The paper's 640^3 density grid in one FP32-mixed evaluation: the density
    # is the 4 x 4 x 4 supercell of a 160^3 system, so E(640^3) = 64 E(160^3)
    # and the potentials are the small system's, tiled (extensivity of the
    # periodic energy); the 160^3 reference is the FP64 form.
    s = _shell160()
    n, sg = s.n.cpu().numpy(), s.sigma.cpu().numpy()
    f = B.Functional(s.shape, s.cell, 1, B.FP64)
    try:
        e64, dn64, ds64 = f.calculate(n, sg)
    finally:
        f.close()
    nb, sgb = np.tile(n, (4, 4, 4)), np.tile(sg, (4, 4, 4))
    f = B.Functional((640, 640, 640), 4 * s.cell, 1, B.FP32_MIXED)
    try:
        e, dn, ds = f.calculate(nb, sgb)
    finally:
        f.close()
    assert abs(e / 64 - e64) <= 1e-6, (e / 64, e64)
    assert np.max(np.abs(dn - np.tile(dn64, (4, 4, 4)))) <= 1e-5 * np.max(np.abs(dn64))
    assert np.max(np.abs(ds - np.tile(ds64, (4, 4, 4)))) <= 1e-5 * np.max(np.abs(ds64))
