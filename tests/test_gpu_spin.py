"""Spin-polarised form (svdW-DF) on the GPU against the spin oracle, both
precisions; its unpolarised limit against the plain form; plain and spin
calls alternating on one handle; host and device forms alike.

Tolerances as for the plain form: FP64, energy 1e-10 relative and each
potential 1e-9 of its max norm; FP32-mixed, |dE| <= 1e-6 Ha and 1e-5 of the
max norm (q0 is FP64 in both)."""
import numpy as np
import pytest

from oracle import spin as ospin
from paper_1703_06999_gb300 import inputs

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1703_06999_gb300.binding")
torch = pytest.importorskip("torch")

TOL = {0: (1e-10, 1e-9), 1: (1e-6, 1e-5)}


def _system(shape, seed, functional, triclinic=False):
    g = np.random.default_rng(seed)
    L = np.array(shape) * g.uniform(0.2, 0.3)
    cell = np.diag(L)
    if triclinic:
        cell = np.array([[L[0], 0, 0], [0.7, L[1], 0], [-0.4, 0.5, L[2]]])
    atoms = [(float(g.uniform(1, 6)), float(g.uniform(1, 2.5)), tuple(g.uniform(0, 1, 3) @ cell))
             for _ in range(5)]
    return inputs.make_system(shape, cell, atoms, functional)


def _check(res, ref, prec):
    e, dn, ds = res
    re, rdn, rds = ref
    etol, ptol = TOL[prec]
    if prec == 0:
        assert abs(e - re) <= etol * max(abs(re), 1e-3), (e, re)
    else:
        assert abs(e - re) <= etol, (e, re)
    for a, b in list(zip(dn, rdn)) + list(zip(ds, rds)):
        assert np.max(np.abs(a - b)) <= ptol * max(np.max(np.abs(b)), 1e-300)


CASES = [("cubic24", (24, 24, 24), 1, False, False), ("tric_28_20_30", (28, 20, 30), 2, True, False),
         ("half_polarised", (20, 24, 18), 1, False, True)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,shape,functional,triclinic,empty", CASES)
def test_spin_matches_oracle(name, shape, functional, triclinic, empty, prec, oracle_default):
    s = _system(shape, 40 + len(name), functional, triclinic)
    nu, nd, su, sd = [x.numpy() for x in inputs.spin_split(s, 0.7, seed=3, empty_down_slab=empty)]
    f = B.Functional(s.shape, s.cell, s.functional, prec)
    try:
        res = f.calculate_spin(nu, nd, su, sd)
    finally:
        f.close()
    ref = ospin.energy_potential_spin(oracle_default, nu, nd, su, sd, s.cell, s.functional)
    _check(res, ref, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_unpolarised_spin_input_gives_the_plain_form(prec):
    s = _system((24, 20, 28), 12, 2)
    n, sg = s.n.numpy(), s.sigma.numpy()
    f = B.Functional(s.shape, s.cell, s.functional, prec)
    try:
        e0, dn0, ds0 = f.calculate(n, sg)
        e, dn, ds = f.calculate_spin(n / 2, n / 2, sg / 4, sg / 4)
        e1, dn1, ds1 = f.calculate(n, sg)                  # the plain form again on the same handle
    finally:
        f.close()
    assert e1 == e0 and np.array_equal(dn1, dn0) and np.array_equal(ds1, ds0)
    # FP64: the same q0 to rounding.  FP32-mixed: the plain q0 is double-float
    # and the plain potential is assembled in FP32, the spin one in FP64
    etol, ptol = (1e-12, 1e-10) if prec == 0 else (1e-9, 1e-5)
    assert abs(e - e0) <= etol * abs(e0) + 1e-15
    for x in dn:
        assert np.max(np.abs(x - dn0)) <= ptol * np.max(np.abs(dn0))
    for x in ds:
        assert np.max(np.abs(x - 2 * ds0)) <= ptol * np.max(np.abs(ds0))


def test_spin_device_form_equals_host_form_and_repeats():
    s = _system((20, 20, 24), 21, 1)
    arrs = [x.numpy() for x in inputs.spin_split(s, 0.5, seed=5)]
    f = B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED)
    try:
        e, dn, ds = f.calculate_spin(*arrs)
        dev = [torch.from_numpy(x).to("cuda:0") for x in arrs]
        out = [torch.empty_like(dev[0]) for _ in range(4)]
        en = torch.zeros(1, dtype=torch.float64, device="cuda:0")
        for _ in range(2):
            B.vdwgb_calculate_spin_device(f.h, *dev, *out, en, torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            B.vdwgb_device_status(0)
            assert float(en[0]) == e
            for a, b in zip(out, list(dn) + list(ds)):
                assert np.array_equal(a.cpu().numpy(), b)
    finally:
        f.close()


def test_spin_rejects_null_arrays():
    s = _system((16, 16, 16), 2, 1)
    f = B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED)
    try:
        x = np.zeros(s.shape)
        with pytest.raises(B.VdwgbError) as ei:
            B.vdwgb_calculate_spin(f.h, x, None, x, x, x, x, x, x)
        assert ei.value.code == -1
    finally:
        f.close()
