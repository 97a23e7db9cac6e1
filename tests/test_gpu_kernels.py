"""A caller's convolution kernel through the same engine (vdwgb_set_kernel_k):
the vdW-DF table handed in explicitly reproduces the built-in one bit for
bit; a Gaussian kernel and a smoothed vdW-DF kernel match the oracle run with
the same table, in both precisions (tolerances as for the plain form)."""
import numpy as np
import pytest

from oracle import vdw
from paper_1703_06999_gb300 import inputs

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1703_06999_gb300.binding")

TOL = {0: (1e-10, 1e-9), 1: (1e-6, 1e-5)}


def _system(shape=(24, 20, 28), seed=3, functional=1):
    g = np.random.default_rng(seed)
    L = np.array(shape) * 0.3
    cell = np.array([[L[0], 0, 0], [0.5, L[1], 0], [-0.3, 0.4, L[2]]])
    atoms = [(float(g.uniform(1, 6)), float(g.uniform(1, 2.5)), tuple(g.uniform(0, 1, 3) @ cell)) for _ in range(4)]
    return inputs.make_system(shape, cell, atoms, functional)


def _tables(oracle_default):
    k = vdw.k_grid(vdw.Params())
    gauss = np.tile(np.exp(-0.5 * k * k), (210, 1))
    smooth = oracle_default.phik * np.exp(-(k / 3.0) ** 2)[None, :]
    return {"gaussian": gauss, "smoothed_vdw": smooth}


def _check(res, ref, prec):
    e, dn, ds = res
    etol, ptol = TOL[prec]
    scale = max(abs(ref.energy), 1e-3) if prec == 0 else 1.0
    assert abs(e - ref.energy) <= etol * scale, (e, ref.energy)
    assert np.max(np.abs(dn - ref.dedn)) <= ptol * np.max(np.abs(ref.dedn))
    sd = np.max(np.abs(ref.dedsigma))
    if sd > 1e-12 * np.max(np.abs(ref.dedn)):      # else dE/dsigma vanishes by construction (checked apart)
        assert np.max(np.abs(ds - ref.dedsigma)) <= ptol * sd


@pytest.mark.parametrize("prec", [1, 0])
def test_vdw_table_handed_in_equals_the_builtin(prec):
    s = _system()
    phik, _, _ = B.vdwgb_kernel_table(0)
    f0 = B.Functional(s.shape, s.cell, s.functional, prec)
    f1 = B.Functional(s.shape, s.cell, s.functional, prec, kernel_k=phik)
    try:
        a = f0.calculate(s.n.numpy(), s.sigma.numpy())
        b = f1.calculate(s.n.numpy(), s.sigma.numpy())
    finally:
        f0.close()
        f1.close()
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("name", ["gaussian", "smoothed_vdw"])
def test_caller_kernel_matches_oracle(name, prec, oracle_default):
    tab = _tables(oracle_default)[name]
    s = _system(seed=5, functional=2)
    f = B.Functional(s.shape, s.cell, s.functional, prec, kernel_k=tab)
    try:
        res = f.calculate(s.n.numpy(), s.sigma.numpy())
        again = f.calculate(s.n.numpy(), s.sigma.numpy())
    finally:
        f.close()
    assert res[0] == again[0]
    ref = vdw.Oracle(vdw.Params(), phik=tab).energy_potential(s.n.numpy(), s.sigma.numpy(), s.cell, s.functional)
    _check(res, ref, prec)
    if name == "gaussian" and prec == 0:
        # partition of unity: every F_a is the same convolution, so dE/dsigma
        # vanishes (in FP32 its rounding residual scales with dq0/dsigma)
        assert np.max(np.abs(res[2])) <= 1e-10 * np.max(np.abs(res[1]))


def test_kernel_table_rules(oracle_default):
    s = _system((16, 16, 16))
    tab = _tables(oracle_default)["gaussian"]
    fa = B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED, kernel_k=tab)
    fb = B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED)
    try:
        with pytest.raises(B.VdwgbError) as ei:
            B.vdwgb_set_kernel_k(fa.h, tab)            # after init
        assert ei.value.code == -4
        with pytest.raises(B.VdwgbError) as ei:
            B.vdwgb_batch_new([fa.h, fb.h])            # different tables do not batch
        assert ei.value.code == -1
    finally:
        fa.close()
        fb.close()
