"""Slab decomposition (the paper's parallel layout, Sec. 3) on one GPU: P
virtual ranks, each with its own slab handle and buffers, whose all-to-all
exchanges are device copies between the ranks' buffers.  Potentials must
equal those of one handle on the whole grid bit for bit (every transform
line and k-point goes through the same arithmetic), the energy up to the
order of its sum; one case also against the oracle."""
import numpy as np
import pytest

from paper_1703_06999_gb300 import inputs

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1703_06999_gb300.binding")
torch = pytest.importorskip("torch")


def _system(shape, seed, functional=1, triclinic=False):
    g = np.random.default_rng(seed)
    L = np.array(shape) * g.uniform(0.2, 0.3)
    cell = np.diag(L)
    if triclinic:
        cell = np.array([[L[0], 0, 0], [0.8, L[1], 0], [-0.5, 0.6, L[2]]])
    atoms = [(float(g.uniform(1, 6)), float(g.uniform(1, 2.5)), tuple(g.uniform(0, 1, 3) @ cell))
             for _ in range(4)]
    return inputs.make_system(shape, cell, atoms, functional)


def _virtual_ranks(s, P, prec):
    """One evaluation of system s split over P virtual ranks on cuda:0."""
    from paper_1703_06999_gb300.slab import LibraryStages
    st = LibraryStages(0)
    nx = s.shape[0]
    nxl = nx // P
    nbytes = st.slab_bytes(s.shape, P, prec)
    assert nbytes > 0
    part = nbytes // P
    rho = s.n.to("cuda:0")
    sig = s.sigma.to("cuda:0")
    ranks = []
    try:
        for r in range(P):
            a, b, x = st.buffer(nbytes), st.buffer(nbytes), st.buffer(nbytes)
            h = st.new(s.functional, s.shape, s.cell, P, r, prec, a, b)
            ranks.append(dict(h=h, a=a, b=b, x=x, e=st.energy_buffer(),
                              dn=torch.empty((nxl,) + s.shape[1:], dtype=torch.float64, device="cuda:0"),
                              ds=torch.empty((nxl,) + s.shape[1:], dtype=torch.float64, device="cuda:0")))
        for r, R in enumerate(ranks):
            st.forward(R["h"], rho[r * nxl:(r + 1) * nxl].contiguous(), sig[r * nxl:(r + 1) * nxl].contiguous())
            st.pack(R["h"], R["x"])
        for r, R in enumerate(ranks):            # forward exchange: part r of every sender
            for q, Q in enumerate(ranks):
                R["b"][q * part:(q + 1) * part].copy_(Q["x"][r * part:(r + 1) * part])
        for R in ranks:
            st.contract(R["h"], R["e"])
        for r, R in enumerate(ranks):            # back: part r of every ky-slab
            for q, Q in enumerate(ranks):
                R["x"][q * part:(q + 1) * part].copy_(Q["b"][r * part:(r + 1) * part])
        for R in ranks:
            st.unpack(R["h"], R["x"])
            st.inverse(R["h"], R["dn"], R["ds"])
        torch.cuda.synchronize()
        st.status()
        parts = [float(R["e"][0]) for R in ranks]
        dn = torch.cat([R["dn"] for R in ranks]).cpu().numpy()
        ds = torch.cat([R["ds"] for R in ranks]).cpu().numpy()
        return sum(parts), dn, ds, parts
    finally:
        for R in ranks:
            st.free(R["h"])


def _whole(s, prec):
    f = B.Functional(s.shape, s.cell, s.functional, prec)
    try:
        return f.calculate(s.n.numpy(), s.sigma.numpy())
    finally:
        f.close()


CASES = [((24, 20, 18), 1, 2, False), ((24, 20, 18), 1, 4, False), ((32, 24, 20), 2, 4, True),
         ((20, 24, 30), 2, 2, True), ((16, 16, 16), 1, 1, False), ((48, 40, 36), 1, 8, False)]


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shape,functional,P,triclinic", CASES)
def test_slab_ranks_equal_one_handle(shape, functional, P, triclinic, prec):
    s = _system(shape, 500 + sum(shape) + P, functional, triclinic)
    e, dn, ds, parts = _virtual_ranks(s, P, prec)
    e1, dn1, ds1 = _whole(s, prec)
    assert abs(e - e1) <= 1e-12 * abs(e1) + 1e-15, (e, e1, parts)
    assert np.array_equal(dn, dn1), np.max(np.abs(dn - dn1))
    assert np.array_equal(ds, ds1), np.max(np.abs(ds - ds1))


def test_slab_ranks_match_oracle(oracle_default):
    s = _system((24, 20, 18), 77, 2, True)
    for prec, etol, ptol in ((0, 1e-10, 1e-9), (1, 1e-6, 1e-5)):
        e, dn, ds, _ = _virtual_ranks(s, 4, prec)
        ref = oracle_default.energy_potential(s.n.numpy(), s.sigma.numpy(), s.cell, s.functional)
        scale = max(abs(ref.energy), 1e-3) if prec == 0 else 1.0
        assert abs(e - ref.energy) <= etol * scale, (prec, e, ref.energy)
        assert np.max(np.abs(dn - ref.dedn)) <= ptol * np.max(np.abs(ref.dedn))
        assert np.max(np.abs(ds - ref.dedsigma)) <= ptol * np.max(np.abs(ref.dedsigma))


def test_slab_evaluator_single_rank():
    # no process group: one rank, the exchanges are copies
    from paper_1703_06999_gb300.slab import SlabEvaluator
    s = _system((24, 20, 18), 91, 1)
    ev = SlabEvaluator(s.shape, s.cell, s.functional, B.FP32_MIXED)
    try:
        dn = torch.empty(s.shape, dtype=torch.float64, device="cuda:0")
        ds = torch.empty_like(dn)
        e = ev.calculate(s.n.to("cuda:0"), s.sigma.to("cuda:0"), dn, ds)
        e2 = ev.calculate(s.n.to("cuda:0"), s.sigma.to("cuda:0"), dn, ds)    # handle reusable
    finally:
        ev.close()
    e1, dn1, ds1 = _whole(s, B.FP32_MIXED)
    assert e == e2 and abs(e - e1) <= 1e-12 * abs(e1)
    assert np.array_equal(dn.cpu().numpy(), dn1) and np.array_equal(ds.cpu().numpy(), ds1)


def test_slab_rejects_bad_decompositions():
    from paper_1703_06999_gb300.slab import LibraryStages
    st = LibraryStages(0)
    assert st.slab_bytes((24, 20, 18), 3, B.FP32_MIXED) == 0      # ny = 20 not a multiple of 3
    assert st.slab_bytes((20, 24, 18), 8, B.FP32_MIXED) == 0      # nx = 20 not a multiple of 8
    buf = st.buffer(st.slab_bytes((24, 20, 18), 2, B.FP32_MIXED))
    with pytest.raises(B.VdwgbError) as ei:
        st.new(1, (24, 20, 18), np.eye(3) * 5, 2, 2, B.FP32_MIXED, buf, buf)   # rank 2 of 2
    assert ei.value.code == -1
    with pytest.raises(B.VdwgbError) as ei:
        st.new(1, (24, 20, 18), np.eye(3) * 5, 3, 0, B.FP32_MIXED, buf, buf)
    assert ei.value.code == -1
