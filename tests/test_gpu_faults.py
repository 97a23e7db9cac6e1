"""GPU: the library's error paths, driven by host-side fault injection
(vdwgb_inject_fault), with no fault of the GPU itself.

* An allocation the library needs fails (as when the device is out of
  memory): the call returns VDWGB_ENOMEM, frees what it had, and the next
  call works.
* A kernel's bounded wait runs out: emulated by setting the device's status
  flag before the host checks it (exactly what such a kernel leaves behind);
  the call returns VDWGB_ETIMEDOUT, the flag is cleared, and the next call
  gives the clean result bit for bit.
Both through a handle, a batch and the server."""
import numpy as np
import pytest

from paper_1703_06999_gb300 import inputs

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1703_06999_gb300.binding")

ENOMEM, ETIMEDOUT = -2, -5


@pytest.fixture(autouse=True)
def disarm():
    B.vdwgb_inject_fault(B.FAULT_NONE)
    yield
    B.vdwgb_inject_fault(B.FAULT_NONE)


def _system():
    return inputs.make_system((24, 20, 18), np.diag([8.0, 7.0, 6.5]), [(3.0, 1.4, (3.0, 3.0, 3.0))], 1)


@pytest.mark.parametrize("prec", [0, 1])
def test_allocation_failure_at_init_then_recovery(prec):
    s = _system()
    B.vdwgb_inject_fault(B.FAULT_ALLOC, 1)
    with pytest.raises(B.VdwgbError) as ei:
        B.Functional(s.shape, s.cell, s.functional, prec)
    assert ei.value.code == ENOMEM
    f = B.Functional(s.shape, s.cell, s.functional, prec)     # nothing left armed
    try:
        e, dn, ds = f.calculate(s.n.numpy(), s.sigma.numpy())
        assert np.isfinite(e)
    finally:
        f.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_timed_out_wait_is_reported_then_cleared(prec):
    s = _system()
    n, sg = s.n.numpy(), s.sigma.numpy()
    f = B.Functional(s.shape, s.cell, s.functional, prec)
    try:
        clean = f.calculate(n, sg)
        B.vdwgb_inject_fault(B.FAULT_WAIT, 1)
        with pytest.raises(B.VdwgbError) as ei:
            f.calculate(n, sg)
        assert ei.value.code == ETIMEDOUT
        B.vdwgb_device_status(0)                               # the flag was cleared
        again = f.calculate(n, sg)
        assert again[0] == clean[0] and np.array_equal(again[1], clean[1]) and np.array_equal(again[2], clean[2])
    finally:
        f.close()


def test_batch_paths_report_both_faults():
    systems = [_system(), inputs.small_cubic(3, ngrid=16)]
    fs = [B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED) for s in systems]
    try:
        B.vdwgb_inject_fault(B.FAULT_ALLOC, 1)
        with pytest.raises(B.VdwgbError) as ei:
            B.vdwgb_batch_new([f.h for f in fs])
        assert ei.value.code == ENOMEM
        bt = B.vdwgb_batch_new([f.h for f in fs])
        try:
            hn = [s.n.numpy().copy() for s in systems]
            hs = [s.sigma.numpy().copy() for s in systems]
            outs = lambda: ([np.empty_like(x) for x in hn], [np.empty_like(x) for x in hn])
            dn, ds = outs()
            clean = B.vdwgb_batch_calculate(bt, hn, hs, dn, ds)
            B.vdwgb_inject_fault(B.FAULT_WAIT, 1)
            dn2, ds2 = outs()
            with pytest.raises(B.VdwgbError) as ei:
                B.vdwgb_batch_calculate(bt, hn, hs, dn2, ds2)
            assert ei.value.code == ETIMEDOUT
            dn3, ds3 = outs()
            again = B.vdwgb_batch_calculate(bt, hn, hs, dn3, ds3)
            assert np.array_equal(again, clean)
        finally:
            B.vdwgb_batch_free(bt)
    finally:
        for f in fs:
            f.close()


def test_server_fails_only_the_faulted_requests():
    s = _system()
    n, sg = s.n.numpy(), s.sigma.numpy()
    f = B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED)
    want = f.calculate(n, sg)
    f.close()
    sv = B.vdwgb_server_new(0, B.FP32_MIXED, pool_bytes=1 << 30, max_batch=1, max_inflight=1)
    try:
        def run():
            dn, ds = np.empty_like(n), np.empty_like(n)
            rid = B.vdwgb_server_submit(sv, s.functional, s.shape, s.cell, n, sg, dn, ds)
            e, _ = B.vdwgb_server_wait(sv, rid, 60.0)
            return e, dn, ds
        B.vdwgb_inject_fault(B.FAULT_ALLOC, 1)                 # the request's plan cannot be allocated
        with pytest.raises(B.VdwgbError) as ei:
            run()
        assert ei.value.code == ENOMEM
        e, dn, ds = run()                                      # the next request is planned and served
        assert e == want[0] and np.array_equal(dn, want[1])
        B.vdwgb_inject_fault(B.FAULT_WAIT, 1)                  # its batch's wait runs out
        with pytest.raises(B.VdwgbError) as ei:
            run()
        assert ei.value.code == ETIMEDOUT
        e, dn, ds = run()                                      # a fresh plan, the same result
        assert e == want[0] and np.array_equal(dn, want[1]) and np.array_equal(ds, want[2])
        st = B.vdwgb_server_stats(sv)
        assert st["failed"] == 2 and st["completed"] == 2
    finally:
        B.vdwgb_server_free(sv)
