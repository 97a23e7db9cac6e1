"""GPU: the batch calls against single evaluations, bit for bit.

A system's arithmetic does not depend on the systems beside it, so the
host-array batch call (vdwgb_batch_calculate, parts pipelined on their own
streams), the device-pointer call (captured graph, independent parts)
and the unsplit batch (VDWGB_BATCH_SPLIT=0) must all reproduce each system's
single evaluation exactly, in both precisions, on repeated calls and when
the two paths alternate on one batch; with 2 and 4 parts, and with the
default split (six parts of one or two systems)."""
import os

import numpy as np
import pytest

from paper_1703_06999_gb300 import inputs

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1703_06999_gb300.binding")


def _systems():
    return [inputs.small_cubic(1, ngrid=24),
            inputs.make_system((20, 24, 30), np.diag([7.0, 8.0, 9.5]), [(3.0, 1.4, (3.0, 4.0, 5.0))], 2),
            inputs.make_system((15, 21, 35), np.diag([6.0, 8.0, 11.0]), [(4.0, 1.2, (3.0, 4.0, 5.0))], 1),
            inputs.small_cubic(4, ngrid=32, functional=2)]


@pytest.fixture(scope="module")
def table():
    return B.vdwgb_kernel_table(0)


def _seven_systems():
    """Seven small systems: the default split cuts them into six parts of one
    or two systems."""
    return [inputs.small_cubic(10 + i, ngrid=(16, 20, 24)[i % 3], functional=1 + i % 2) for i in range(7)]


@pytest.mark.parametrize("split,systems_of,parts", [("2", _systems, 2), ("4", _systems, 4), ("0", _systems, 1),
                                                    (None, _seven_systems, 6)],
                         ids=["split2", "split4", "unsplit", "default_split"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_batch_paths_match_single_evaluations(table, prec, split, systems_of, parts):
    import torch
    systems = systems_of()
    fs = [B.Functional(s.shape, s.cell, s.functional, prec) for s in systems]
    old = os.environ.get("VDWGB_BATCH_SPLIT")
    if split is None:
        os.environ.pop("VDWGB_BATCH_SPLIT", None)
    else:
        os.environ["VDWGB_BATCH_SPLIT"] = split
    bt = None
    try:
        alone = [f.calculate(s.n.numpy(), s.sigma.numpy()) for f, s in zip(fs, systems)]
        bt = B.vdwgb_batch_new([f.h for f in fs])
        hn = [s.n.numpy().copy() for s in systems]
        hs = [s.sigma.numpy().copy() for s in systems]
        for rep in range(2):
            hdn = [np.full_like(x, np.nan) for x in hn]
            hds = [np.full_like(x, np.nan) for x in hn]
            e = B.vdwgb_batch_calculate(bt, hn, hs, hdn, hds)
            for i, (ea, dna, dsa) in enumerate(alone):
                assert e[i] == ea, (rep, i)
                assert np.array_equal(hdn[i], dna), (rep, i)
                assert np.array_equal(hds[i], dsa), (rep, i)
        # the device-pointer (graph) path on the same batch, then the host path again
        dev = torch.device("cuda:0")
        ns = [s.n.to(dev) for s in systems]
        ss = [s.sigma.to(dev) for s in systems]
        dn = [torch.empty_like(x) for x in ns]
        ds = [torch.empty_like(x) for x in ns]
        en = torch.zeros(len(fs), dtype=torch.float64, device=dev)
        B.vdwgb_batch_calculate_device(bt, ns, ss, dn, ds, en, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        for i, (ea, dna, dsa) in enumerate(alone):
            assert float(en[i]) == ea
            assert np.array_equal(dn[i].cpu().numpy(), dna)
            assert np.array_equal(ds[i].cpu().numpy(), dsa)
        hdn = [np.full_like(x, np.nan) for x in hn]
        hds = [np.full_like(x, np.nan) for x in hn]
        e = B.vdwgb_batch_calculate(bt, hn, hs, hdn, hds)
        assert all(e[i] == alone[i][0] for i in range(len(fs)))
        assert all(np.array_equal(hdn[i], alone[i][1]) for i in range(len(fs)))
        assert B.vdwgb_batch_launches(bt) == 8 * parts
    finally:
        if bt is not None:
            B.vdwgb_batch_free(bt)
        if old is None:
            os.environ.pop("VDWGB_BATCH_SPLIT", None)
        else:
            os.environ["VDWGB_BATCH_SPLIT"] = old
        for f in fs:
            f.close()
