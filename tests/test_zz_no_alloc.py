"""GPU: the allocation-free entry point (vdwgb_calculate_noalloc) against the
handle path (vdwgb_calculate_device, FP32-mixed, cubic) on the same inputs.

Both compute the same FP32-mixed arithmetic, so they must agree within the
FP32-mixed test tolerance: |dE| <= 1e-6 Ha, potential max-norm error <= 1e-5
relative.  Each case runs twice in a row with another grid in between, since
all calls share one fixed scratch array."""
import numpy as np
import pytest

from paper_1703_06999_gb300 import inputs

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1703_06999_gb300.binding")

ETOL, PTOL = 1e-6, 1e-5

CASES = [
    ("cubic24", lambda: inputs.small_cubic(4, ngrid=24)),
    ("ragged", lambda: inputs.make_system((20, 24, 30), np.diag([7.0, 8.0, 9.5]), [(3.0, 1.4, (3.0, 4.0, 5.0))], 2)),
    ("odd357", lambda: inputs.make_system((15, 21, 35), np.diag([6.0, 8.0, 11.0]), [(4.0, 1.2, (3.0, 4.0, 5.0))], 1)),
    ("triclinic", lambda: inputs.make_system((16, 18, 20),
                                             np.array([[7.0, 0, 0], [1.5, 6.5, 0], [-0.8, 1.1, 7.2]]),
                                             [(2.0, 1.3, (3.0, 3.0, 3.0)), (6.0, 2.5, (5.0, 2.0, 4.0))], 1)),
    ("thin", lambda: inputs.make_system((2, 3, 64), np.diag([1.0, 1.5, 20.0]), [(1.0, 1.0, (0.5, 0.5, 10.0))], 2)),
    ("max32", lambda: inputs.make_system((32, 32, 32), np.diag([10.0, 10.0, 10.0]),
                                         [(3.0, 1.5, (3.0, 3.0, 3.0)), (6.5, 2.0, (6.0, 7.0, 5.0))], 1)),
]


@pytest.fixture(scope="module")
def dev():
    import torch
    B.vdwgb_kernel_table(0)       # the table must be resident before the first call
    return torch.device("cuda:0")


def _to(dev, s):
    return s.n.to(dev).contiguous(), s.sigma.to(dev).contiguous()


def _noalloc(dev, s, n, sg):
    import torch
    dn = torch.full_like(n, float("nan"))
    ds = torch.full_like(n, float("nan"))
    e = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    B.vdwgb_calculate_noalloc(0, s.functional, s.shape, s.cell, n, sg, dn, ds, e,
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    B.vdwgb_device_status(0)       # raises if a bounded wait ran out (results invalid)
    return float(e[0]), dn.cpu().numpy(), ds.cpu().numpy()


def _handle(dev, s, n, sg):
    import torch
    f = B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED)
    try:
        dn = torch.empty_like(n)
        ds = torch.empty_like(n)
        e = torch.zeros(1, dtype=torch.float64, device=dev)
        f.calculate_device(n, sg, dn, ds, e, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        return float(e[0]), dn.cpu().numpy(), ds.cpu().numpy()
    finally:
        f.close()


def _close(a, b):
    ea, dna, dsa = a
    eb, dnb, dsb = b
    assert np.isfinite(ea) and np.all(np.isfinite(dna)) and np.all(np.isfinite(dsa))
    assert abs(ea - eb) <= ETOL, (ea, eb)
    assert np.max(np.abs(dna - dnb)) <= PTOL * max(np.max(np.abs(dnb)), 1e-300)
    assert np.max(np.abs(dsa - dsb)) <= PTOL * max(np.max(np.abs(dsb)), 1e-300)


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_handle_path_twice(dev, name, make):
    s = make()
    other = inputs.small_cubic(9, ngrid=20)
    n, sg = _to(dev, s)
    on, osg = _to(dev, other)
    want = _handle(dev, s, n, sg)
    first = _noalloc(dev, s, n, sg)
    _close(first, want)
    _noalloc(dev, other, on, osg)          # leaves a different grid's data in the scratch
    second = _noalloc(dev, s, n, sg)
    _close(second, want)
    third = _noalloc(dev, s, n, sg)        # directly after itself
    _close(third, want)


@pytest.mark.parametrize("shape", [(65, 8, 8), (40, 40, 40), (64, 64, 16), (11, 8, 8), (0, 8, 8)])
def test_noalloc_rejects_beyond_limits(dev, shape):
    import torch
    npts = max(shape[0] * shape[1] * shape[2], 1)
    n = torch.full((npts,), 0.01, dtype=torch.float64, device=dev)
    out = torch.empty_like(n)
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(B.VdwgbError) as ei:
        B.vdwgb_calculate_noalloc(0, B.DF1, shape, np.diag([8.0, 8.0, 8.0]), n, n, out, out, e, 0)
    assert ei.value.code == -1


def test_noalloc_refuses_a_capturing_stream(dev):
    # the plan data are copied from pageable host memory: the call cannot be
    # captured and must say so instead of recording those copies
    import torch
    s = inputs.small_cubic(4, ngrid=16)
    n, sg = _to(dev, s)
    out = torch.empty_like(n)
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    code = None
    with torch.cuda.graph(g, stream=st):
        try:
            B.vdwgb_calculate_noalloc(0, s.functional, s.shape, s.cell, n, sg, out, out, e, st.cuda_stream)
        except B.VdwgbError as err:
            code = err.code
        e.add_(0.0)                # keep the captured graph non-empty
    assert code == -4
    torch.cuda.synchronize()
    _close(_noalloc(dev, s, n, sg), _handle(dev, s, n, sg))   # the array is still usable
