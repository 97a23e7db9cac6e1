"""GPU: the cluster plane kernel (y / x transforms, contraction and inverses
of each kz-plane in one 16-CTA cluster, opt-in) against the separate passes
and the FP64 oracle, on grids whose x and y lengths it accepts.

Tolerances as for the FP32-mixed path: |dE| <= 1e-6 Ha and potential
max-norm error <= 1e-5 relative against the oracle; the two GPU paths differ
only in FP32 rounding order."""
import numpy as np
import pytest

from paper_1703_06999_gb300 import inputs

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1703_06999_gb300.binding")

CASES = [
    ("c16", lambda: inputs.make_system((16, 16, 24), np.diag([6.0, 6.0, 8.0]), [(3.0, 1.5, (3.0, 3.0, 4.0))], 1)),
    ("c32", lambda: inputs.small_cubic(3, ngrid=32)),
    ("tric48_32_40", lambda: inputs.make_system((48, 32, 40), np.array([[9.0, 0, 0], [1.5, 6.5, 0], [-0.8, 1.1, 7.2]]),
                                                [(2.0, 1.3, (3.0, 3.0, 3.0)), (6.0, 2.5, (5.0, 2.0, 4.0))], 2)),
    ("c64_80_112", lambda: inputs.make_system((64, 80, 112), np.diag([12.0, 15.0, 20.0]),
                                              [(3.0, 1.5, (6.0, 7.0, 9.0)), (5.0, 2.0, (5.0, 8.0, 12.0))], 1)),
]


def _run(s, fused):
    B.vdwgb_set_fused(fused)
    try:
        f = B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED)
    finally:
        B.vdwgb_set_fused(0)
    try:
        info = B.vdwgb_plan_info(f.h)
        e, dn, ds = f.calculate(s.n.numpy(), s.sigma.numpy())
        return info, (e, dn, ds)
    finally:
        f.close()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_plane_kernel_matches_oracle_and_separate_passes(oracle_default, name, make):
    s = make()
    ref = oracle_default.energy_potential(s.n.numpy(), s.sigma.numpy(), s.cell, s.functional)
    info_f, (ef, dnf, dsf) = _run(s, 1)
    info_s, (es, dns, dss) = _run(s, 0)
    assert info_f["cluster"] == 16 and info_s["cluster"] == 0
    assert info_f["launches"] == 4 and info_s["launches"] == 8
    for e, dn, ds in ((ef, dnf, dsf), (es, dns, dss)):
        assert abs(e - ref.energy) <= 1e-6
        assert np.max(np.abs(dn - ref.dedn)) <= 1e-5 * np.max(np.abs(ref.dedn))
        assert np.max(np.abs(ds - ref.dedsigma)) <= 1e-5 * np.max(np.abs(ref.dedsigma))
    assert abs(ef - es) <= 1e-7 * max(abs(es), 1e-3)


def test_plane_kernel_in_a_mixed_batch(oracle_default):
    """Fused and non-fused systems in one batch: each result equals its
    evaluation alone (the batch runs both the plane kernel and the separate
    passes, each over its own systems)."""
    import torch
    systems = [inputs.small_cubic(3, ngrid=32), inputs.small_cubic(5, ngrid=24),
               inputs.make_system((48, 32, 40), np.diag([9.0, 6.5, 7.2]), [(2.0, 1.3, (3.0, 3.0, 3.0))], 2)]
    B.vdwgb_set_fused(1)
    try:
        fs = [B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED) for s in systems]
    finally:
        B.vdwgb_set_fused(0)
    try:
        assert [B.vdwgb_plan_info(f.h)["cluster"] for f in fs] == [16, 0, 16]
        dev = torch.device("cuda:0")
        ns = [s.n.to(dev) for s in systems]
        ss = [s.sigma.to(dev) for s in systems]
        dn = [torch.empty_like(x) for x in ns]
        ds = [torch.empty_like(x) for x in ns]
        en = torch.zeros(len(fs), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        for i, f in enumerate(fs):
            f.calculate_device(ns[i], ss[i], dn[i], ds[i], en[i:i + 1], stream)
        torch.cuda.synchronize()
        alone = [(float(en[i]), dn[i].cpu().numpy(), ds[i].cpu().numpy()) for i in range(len(fs))]
        bt = B.vdwgb_batch_new([f.h for f in fs])
        try:
            # fused and unfused systems together use all nine stage kinds (a
            # batch split into parts launches the stages of each part)
            assert B.vdwgb_batch_launches(bt) >= 9
            en.zero_()
            B.vdwgb_batch_calculate_device(bt, ns, ss, dn, ds, en, stream)
            torch.cuda.synchronize()
            for i in range(len(fs)):
                assert float(en[i]) == alone[i][0]
                assert np.array_equal(dn[i].cpu().numpy(), alone[i][1])
                assert np.array_equal(ds[i].cpu().numpy(), alone[i][2])
        finally:
            B.vdwgb_batch_free(bt)
    finally:
        for f in fs:
            f.close()
