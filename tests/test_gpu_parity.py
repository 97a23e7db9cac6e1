"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances: FP64 path, energy 1e-10 relative and potential 1e-9 of its max
norm (rounding order only); FP32-mixed path, |dE| <= 1e-6 Ha and potential
max-norm error <= 1e-5 relative, the accuracy targets of this workload."""
import numpy as np
import pytest

from oracle import vdw
from paper_1703_06999_gb300 import inputs

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1703_06999_gb300.binding")

TOL = {0: (1e-10, 1e-9), 1: (1e-6, 1e-5)}   # precision -> (energy, potential)


def _check(res_gpu, ref, prec, rel_energy=True):
    e, dn, ds = res_gpu
    etol, ptol = TOL[prec]
    if prec == B.FP64:
        assert abs(e - ref.energy) <= etol * max(abs(ref.energy), 1e-3), (e, ref.energy)
    else:
        assert abs(e - ref.energy) <= etol, (e, ref.energy)
    sn = max(np.max(np.abs(ref.dedn)), 1e-300)
    ss = max(np.max(np.abs(ref.dedsigma)), 1e-300)
    assert np.max(np.abs(dn - ref.dedn)) <= ptol * sn
    assert np.max(np.abs(ds - ref.dedsigma)) <= ptol * ss


@pytest.fixture(scope="module")
def gpu_table():
    return B.vdwgb_kernel_table(0)


def test_kernel_table_matches_oracle(gpu_table, oracle_default):
    phik, phir, q = gpu_table
    p = vdw.Params()
    assert np.allclose(q, vdw.q_mesh(p), rtol=1e-15, atol=0)
    _, phir_o = vdw.kernel_table(p)
    # r = 0 holds phi(0, 0), which is log-divergent and carries zero weight
    scale = np.max(np.abs(phir_o[:, 1:]), axis=1, keepdims=True)
    assert np.max(np.abs(phir[:, 1:] - phir_o[:, 1:]) / scale) < 1e-11
    phik_o = oracle_default.phik
    scale = np.max(np.abs(phik_o), axis=1, keepdims=True)
    assert np.max(np.abs(phik - phik_o) / scale) < 1e-10


def test_phi_points_match_oracle():
    rng = np.random.default_rng(11)
    d1 = np.concatenate([rng.uniform(0, 3, 40), rng.uniform(0, 60, 40), [0.0, 1e-3, 500.0]])
    d2 = np.concatenate([rng.uniform(0, 3, 40), rng.uniform(0, 60, 40), [0.0, 2e-3, 499.0]])
    g = B.vdwgb_phi(d1, d2)
    o = vdw.phi_dion(d1, d2)
    assert np.allclose(g, o, rtol=1e-10, atol=1e-13 * np.max(np.abs(o)))


CASES = [
    ("cubic24", lambda: inputs.small_cubic(0, ngrid=24)),
    ("ragged", lambda: inputs.make_system((30, 20, 18), np.diag([9.0, 7.0, 6.0]),
                                          [(3.0, 1.5, (2.0, 3.0, 1.0)), (5.0, 2.0, (6.0, 4.0, 4.0))], 2)),
    ("odd357", lambda: inputs.make_system((15, 21, 35), np.diag([6.0, 8.0, 11.0]),
                                          [(4.0, 1.2, (3.0, 4.0, 5.0))], 1)),
    ("triclinic", lambda: inputs.make_system((16, 18, 20), np.array([[7.0, 0, 0], [1.5, 6.5, 0], [-0.8, 1.1, 7.2]]),
                                             [(2.0, 1.3, (3.0, 3.0, 3.0)), (6.0, 2.5, (5.0, 2.0, 4.0))], 1)),
    ("thin", lambda: inputs.make_system((2, 3, 64), np.diag([1.0, 1.5, 20.0]),
                                        [(1.0, 1.0, (0.5, 0.5, 10.0))], 1)),
    ("hello", inputs.hello_example),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_end_to_end_matches_oracle(oracle_default, name, make, prec):
    s = make()
    n, sg = s.n.numpy(), s.sigma.numpy()
    ref = oracle_default.energy_potential(n, sg, s.cell, s.functional)
    f = B.Functional(s.shape, s.cell, s.functional, prec)
    try:
        got = f.calculate(n, sg)
        _check(got, ref, prec)
        again = f.calculate(n, sg)
        assert again[0] == got[0] and np.array_equal(again[1], got[1])   # deterministic
    finally:
        f.close()


def test_linear_interpolation_matches_oracle(oracle_linear):
    s = inputs.small_cubic(1, ngrid=24)
    n, sg = s.n.numpy(), s.sigma.numpy()
    ref = oracle_linear.energy_potential(n, sg, s.cell, s.functional)
    f = B.Functional(s.shape, s.cell, s.functional, B.FP64, interp=B.INTERP_LINEAR)
    try:
        _check(f.calculate(n, sg), ref, B.FP64)
    finally:
        f.close()


def test_dimer_96_full_size(oracle_default):
    # the benchmark workload (96^3, 18 x 18 x 24 bohr), both precisions, both functionals
    for fn in (1, 2):
        s = inputs.dimer(0, functional=fn)
        n, sg = s.n.numpy(), s.sigma.numpy()
        ref = oracle_default.energy_potential(n, sg, s.cell, fn)
        for prec in (B.FP64, B.FP32_MIXED):
            f = B.Functional(s.shape, s.cell, fn, prec)
            try:
                _check(f.calculate(n, sg), ref, prec)
            finally:
                f.close()


def test_device_pointer_path_and_batch(oracle_default):
    import torch
    systems = [inputs.small_cubic(2, ngrid=24),
               inputs.make_system((20, 24, 30), np.diag([7.0, 8.0, 9.5]), [(3.0, 1.4, (3.0, 4.0, 5.0))], 2),
               inputs.make_system((32, 16, 24), np.diag([10.0, 5.0, 7.0]), [(2.0, 1.1, (5.0, 2.0, 3.0))], 1)]
    refs = [oracle_default.energy_potential(s.n.numpy(), s.sigma.numpy(), s.cell, s.functional) for s in systems]
    for prec in (B.FP64, B.FP32_MIXED):
        fs = [B.Functional(s.shape, s.cell, s.functional, prec) for s in systems]
        try:
            dev = torch.device("cuda:0")
            ns = [s.n.to(dev) for s in systems]
            ss = [s.sigma.to(dev) for s in systems]
            dn = [torch.empty_like(x) for x in ns]
            ds = [torch.empty_like(x) for x in ns]
            en = torch.zeros(len(systems), dtype=torch.float64, device=dev)
            stream = torch.cuda.current_stream().cuda_stream
            for i, f in enumerate(fs):
                f.calculate_device(ns[i], ss[i], dn[i], ds[i], en[i:i + 1], stream)
            torch.cuda.synchronize()
            alone = [(float(en[i]), dn[i].cpu().numpy(), ds[i].cpu().numpy()) for i in range(len(fs))]
            for a, r in zip(alone, refs):
                _check(a, r, prec)
            bt = B.vdwgb_batch_new([f.h for f in fs])
            try:
                for _ in range(2):   # second call replays the captured graph
                    for x in dn + ds:
                        x.zero_()
                    en.zero_()
                    B.vdwgb_batch_calculate_device(bt, ns, ss, dn, ds, en, stream)
                    torch.cuda.synchronize()
                    for i in range(len(fs)):
                        # a system gives the same result alone and in the batch
                        assert float(en[i]) == alone[i][0]
                        assert np.array_equal(dn[i].cpu().numpy(), alone[i][1])
                        assert np.array_equal(ds[i].cpu().numpy(), alone[i][2])
            finally:
                B.vdwgb_batch_free(bt)
        finally:
            for f in fs:
                f.close()


def test_errors_are_reported():
    h = B.vdwgb_new(1)
    try:
        with pytest.raises(B.VdwgbError):
            B.vdwgb_calculate(h, np.zeros(1), np.zeros(1), np.zeros(1), np.zeros(1))
        with pytest.raises(B.VdwgbError):
            B.vdwgb_init_cuda(h, 0, 7)
        B.vdwgb_set_unit_cell(h, (4, 4, 4), np.eye(3) * 3)
        with pytest.raises(B.VdwgbError):
            B.vdwgb_init_cuda(h, 99, 0)
    finally:
        B.vdwgb_finalize(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_q0_step_matches_oracle(prec):
    # q0 and its derivatives exactly as each form computes them inside the
    # evaluation (FP32-mixed: double-float q0, FP32 derivatives).
    rng = np.random.default_rng(5)
    n = 10 ** rng.uniform(-11, 2, 4000)
    s = 10 ** rng.uniform(-12, 3, 4000) * n ** (8 / 3) * rng.uniform(0, 50, 4000)
    s[:50] = 0.0
    for fn in (1, 2):
        q, dn, ds = B.vdwgb_q0(n, s, fn, prec)
        rq, rdn, rds = vdw.q0_of(n, s, fn)
        assert np.max(np.abs(q - rq) / rq) < (1e-12 if prec == 0 else 1e-11)
        tol = 1e-12 if prec == 0 else 1e-5
        for got, ref in ((dn, rdn), (ds, rds)):
            big = np.abs(ref) > 1e-6 * np.max(np.abs(ref))
            assert np.max(np.abs(got[big] - ref[big]) / np.abs(ref[big])) < tol


def test_autotuned_tiles_give_identical_results():
    # Tile shapes only regroup independent lines and butterflies: the tuned
    # plan must reproduce the default plan bit for bit.
    s = inputs.make_system((40, 36, 30), np.diag([9.0, 8.0, 7.5]), [(3.0, 1.4, (4.0, 3.0, 3.0))], 1)
    n, sg = s.n.numpy(), s.sigma.numpy()
    for prec in (B.FP32_MIXED, B.FP64):
        B.vdwgb_set_autotune(False)
        f0 = B.Functional(s.shape, s.cell, 1, prec)
        r0 = f0.calculate(n, sg)
        f0.close()
        B.vdwgb_set_autotune(True)
        try:
            f1 = B.Functional(s.shape, s.cell, 1, prec)
            info = B.vdwgb_plan_info(f1.h)
            r1 = f1.calculate(n, sg)
            f1.close()
        finally:
            B.vdwgb_set_autotune(False)
        assert info["autotuned"] == 1 and info["launches"] == 8
        assert r1[0] == r0[0] and np.array_equal(r1[1], r0[1]) and np.array_equal(r1[2], r0[2])
