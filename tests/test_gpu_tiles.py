"""GPU: every tile shape a plan can take gives the oracle's result.

vdwgb_set_tiles forces the z-forward / z-inverse lines per tile, the y / x
kz-columns per tile and the y / x ring depths.  The sweep covers tiles wider
than one line per thread of a 256-thread block (20 W or 10 LZ above 256
lines), axes with and without an in-place two-pass split, ragged last tiles
and both precisions.  Shapes beyond shared memory are refused with
VDWGB_EINVAL; the others must match the oracle to the parity tolerances."""
import numpy as np
import pytest

from oracle import vdw
from paper_1703_06999_gb300 import inputs

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1703_06999_gb300.binding")

TOL = {0: (1e-10, 1e-9), 1: (1e-6, 1e-5)}   # precision -> (energy, potential)

GRIDS = [
    # no split on any axis (generic transforms everywhere)
    ("odd", lambda: inputs.make_system((15, 21, 35), np.diag([6.0, 8.0, 11.0]), [(4.0, 1.2, (3.0, 4.0, 5.0))], 1)),
    # split on every axis in FP32 (in-place transforms)
    ("split", lambda: inputs.make_system((24, 16, 48), np.diag([8.0, 6.0, 12.0]),
                                          [(3.0, 1.4, (3.0, 3.0, 5.0)), (5.0, 2.0, (5.0, 3.0, 7.0))], 2)),
    # mixed: split y and z, generic x
    ("mixed", lambda: inputs.make_system((20, 32, 40), np.diag([7.0, 9.0, 10.0]), [(3.0, 1.5, (3.0, 4.0, 5.0))], 1)),
]

# (lz, lzi, wy, wx, nby, nbx)
SHAPES = [
    (1, 1, 1, 1, 1, 1),
    (3, 5, 5, 3, 2, 3),
    (2, 2, 6, 6, 2, 2),
    (8, 8, 8, 8, 4, 4),
    (12, 7, 12, 12, 1, 2),
    (16, 16, 16, 16, 1, 1),      # 320 lines per y / x tile
    (4, 4, 16, 2, 1, 1),         # 320-line y tiles within FP64 shared memory
    (25, 26, 13, 14, 3, 1),      # 250 / 260 z lines, ragged column tiles
    (32, 3, 2, 17, 2, 1),        # 320 z lines per forward tile
]


@pytest.fixture(scope="module")
def table():
    return B.vdwgb_kernel_table(0)


def _close(res, ref, prec):
    e, dn, ds = res
    etol, ptol = TOL[prec]
    if prec == B.FP64:
        assert abs(e - ref.energy) <= etol * max(abs(ref.energy), 1e-3), (e, ref.energy)
    else:
        assert abs(e - ref.energy) <= etol, (e, ref.energy)
    assert np.max(np.abs(dn - ref.dedn)) <= ptol * max(np.max(np.abs(ref.dedn)), 1e-300)
    assert np.max(np.abs(ds - ref.dedsigma)) <= ptol * max(np.max(np.abs(ref.dedsigma)), 1e-300)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name,make", GRIDS, ids=[g[0] for g in GRIDS])
def test_forced_tile_shapes_match_oracle(table, name, make, prec):
    s = make()
    n, sg = s.n.numpy(), s.sigma.numpy()
    ref = vdw.Oracle().energy_potential(n, sg, s.cell, s.functional)
    f = B.Functional(s.shape, s.cell, s.functional, prec)
    ran = 0
    try:
        for shape in SHAPES:
            try:
                B.vdwgb_set_tiles(f.h, *shape)
            except B.VdwgbError as err:
                assert err.code == -1, (shape, err)   # beyond shared memory or range
                continue
            info = B.vdwgb_plan_info(f.h)
            assert (info["LZ"], info["LZi"], info["Wy"], info["Wx"]) == shape[:4]
            assert info["nbuf_yx"] == 10 * shape[4] + shape[5]
            _close(f.calculate(n, sg), ref, prec)
            ran += 1
    finally:
        f.close()
    assert ran >= 3, ran


def test_set_tiles_rejects_bad_shapes_and_held_handles(table):
    s = inputs.small_cubic(2, ngrid=20)
    f = B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED)
    try:
        nzh = s.shape[2] // 2 + 1
        for bad in [(0, 1, 1, 1, 1, 1), (1, 1, nzh + 1, 1, 1, 1), (1, 1, 1, 1, 5, 1),
                    (1, 20 * 20 + 1, 1, 1, 1, 1), (1, 1, 1, 1, 1, 0)]:
            with pytest.raises(B.VdwgbError) as ei:
                B.vdwgb_set_tiles(f.h, *bad)
            assert ei.value.code == -1
        bt = B.vdwgb_batch_new([f.h])
        try:
            with pytest.raises(B.VdwgbError) as ei:
                B.vdwgb_set_tiles(f.h, 2, 2, 2, 2, 2, 2)
            assert ei.value.code == -4
        finally:
            B.vdwgb_batch_free(bt)
        B.vdwgb_set_tiles(f.h, 2, 2, 2, 2, 2, 2)   # allowed again once the batch is gone
        ref = vdw.Oracle().energy_potential(s.n.numpy(), s.sigma.numpy(), s.cell, s.functional)
        _close(f.calculate(s.n.numpy(), s.sigma.numpy()), ref, 1)
    finally:
        f.close()


def test_fp32_interval_decision_random_triclinic_cells(table):
    """The host sorts k-points into kernel-table intervals with the same FP32
    arithmetic as the contraction kernel; a disagreement would surface as a
    VDWGB_ECUDA status from the host-array call.  Random triclinic cells put
    many |k| near interval boundaries."""
    rng = np.random.default_rng(1234)
    for case in range(8):
        shape = tuple(int(v) for v in rng.choice([12, 15, 16, 18, 20, 24], 3))
        a = np.diag(rng.uniform(5.0, 9.0, 3)) + np.tril(rng.uniform(-1.5, 1.5, (3, 3)), -1)
        centre = tuple(a.sum(axis=0) / 2)
        s = inputs.make_system(shape, a, [(3.0, 1.4, centre)], 1 + case % 2)
        n, sg = s.n.numpy(), s.sigma.numpy()
        ref = vdw.Oracle().energy_potential(n, sg, s.cell, s.functional)
        f = B.Functional(s.shape, s.cell, s.functional, B.FP32_MIXED)
        try:
            _close(f.calculate(n, sg), ref, 1)
        finally:
            f.close()
