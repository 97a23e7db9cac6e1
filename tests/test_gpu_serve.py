"""Served form: requests of different grids submitted while others run give
the same result as the same evaluation alone, and match the oracle."""
import numpy as np
import pytest

from oracle import vdw
from paper_1703_06999_gb300 import inputs

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1703_06999_gb300.binding")


def _requests():
    shapes = [(24, 24, 24), (32, 24, 20), (20, 28, 36), (48, 40, 36), (30, 30, 30), (16, 64, 18),
              (40, 36, 32), (24, 20, 60), (36, 36, 36), (28, 42, 30), (50, 20, 24), (64, 32, 24)]
    out = []
    for i, sh in enumerate(shapes):
        g = np.random.default_rng(100 + i)
        h = g.uniform(0.2, 0.3)
        L = np.array(sh) * h
        atoms = [(float(g.uniform(1, 6)), float(g.uniform(1, 2.5)), tuple(g.uniform(0, 1, 3) * L))
                 for _ in range(int(g.integers(2, 8)))]
        out.append(inputs.make_system(sh, np.diag(L), atoms, 1 + i % 2))
    return out


@pytest.mark.parametrize("prec", [1, 0])
def test_served_results_equal_alone_and_oracle(prec, oracle_default):
    systems = _requests()
    alone = []
    for s in systems:
        f = B.Functional(s.shape, s.cell, s.functional, prec)
        alone.append(f.calculate(s.n.numpy(), s.sigma.numpy()))
        f.close()
    sv = B.vdwgb_server_new(0, prec, pool_bytes=1 << 30, max_batch=5, max_inflight=2)
    try:
        outs, ids = [], []
        for rep in range(2):          # every system twice, interleaved with the others
            for s in systems:
                dn = np.empty(s.shape)
                ds = np.empty(s.shape)
                outs.append((s, dn, ds))
                ids.append(B.vdwgb_server_submit(sv, s.functional, s.shape, s.cell, s.n.numpy(), s.sigma.numpy(),
                                                 dn, ds))
        for k, rid in enumerate(ids):
            e, lat = B.vdwgb_server_wait(sv, rid, 120.0)
            s, dn, ds = outs[k]
            a = alone[k % len(systems)]
            assert e == a[0]                      # deterministic: same alone and in any batch
            assert np.array_equal(dn, a[1]) and np.array_equal(ds, a[2])
            assert lat > 0
        st = B.vdwgb_server_stats(sv)
        assert st["completed"] == len(ids) and st["failed"] == 0
        assert st["batches"] >= 1 and st["p99_s"] >= st["p50_s"] > 0
        assert st["pool_used_peak"] <= st["pool_bytes"]
    finally:
        B.vdwgb_server_free(sv)
    # two of them against the oracle
    for s, a in list(zip(systems, alone))[:2]:
        ref = oracle_default.energy_potential(s.n.numpy(), s.sigma.numpy(), s.cell, s.functional)
        etol = 1e-10 * max(1e-3, abs(ref.energy)) if prec == 0 else 1e-6
        assert abs(a[0] - ref.energy) <= etol


def test_server_rejects_oversized_and_bad_requests():
    sv = B.vdwgb_server_new(0, B.FP32_MIXED, pool_bytes=64 << 20, max_batch=2, max_inflight=1)
    try:
        big = np.zeros(1)
        with pytest.raises(B.VdwgbError) as ei:
            B.vdwgb_server_submit(sv, 1, (192, 192, 192), np.eye(3) * 30, big, big, big, big)
        assert ei.value.code == -6      # EAGAIN: footprint exceeds the pool
        x = np.full((11, 4, 4), 0.1)
        ox, oy = np.empty_like(x), np.empty_like(x)      # alive until the request is reported
        rid = B.vdwgb_server_submit(sv, 1, (11, 4, 4), np.eye(3) * 4, x, x, ox, oy)
        with pytest.raises(B.VdwgbError):
            B.vdwgb_server_wait(sv, rid, 30.0)   # prime factor 11: the planner fails the request
        with pytest.raises(B.VdwgbError):
            B.vdwgb_server_poll(sv, 123456)      # unknown id
    finally:
        B.vdwgb_server_free(sv)


@pytest.mark.parametrize("prec", [1, 0])
def test_resident_plans_are_replanned_for_new_cells(prec):
    # Requests of one grid but different cells and functionals, one after the
    # other: from the second on, each re-plans the resident plan of its grid
    # (metric, k-point order sorted on the device, chunks) and must give the
    # result of a fresh handle bit for bit.
    systems = []
    for i in range(6):
        sh = (24, 20, 30) if i % 2 == 0 else (32, 32, 16)
        g = np.random.default_rng(300 + i)
        L = np.array(sh) * g.uniform(0.18, 0.32)
        cell = np.diag(L)
        if i == 4:                                   # a triclinic cell too
            cell = np.array([[L[0], 0, 0], [0.7, L[1], 0], [-0.4, 0.9, L[2]]])
        atoms = [(float(g.uniform(1, 6)), float(g.uniform(1, 2.5)), tuple(g.uniform(0, 1, 3) @ cell))
                 for _ in range(3)]
        systems.append(inputs.make_system(sh, cell, atoms, 1 + (i // 2) % 2))
    alone = []
    for s in systems:
        f = B.Functional(s.shape, s.cell, s.functional, prec)
        alone.append(f.calculate(s.n.numpy(), s.sigma.numpy()))
        f.close()
    sv = B.vdwgb_server_new(0, prec, pool_bytes=1 << 30, max_batch=4, max_inflight=2)
    try:
        for s, a in zip(systems, alone):
            dn, ds = np.empty(s.shape), np.empty(s.shape)
            rid = B.vdwgb_server_submit(sv, s.functional, s.shape, s.cell, s.n.numpy(), s.sigma.numpy(), dn, ds)
            e, _ = B.vdwgb_server_wait(sv, rid, 120.0)
            assert e == a[0] and np.array_equal(dn, a[1]) and np.array_equal(ds, a[2])
        st = B.vdwgb_server_stats(sv)
        assert st["plans_built"] == 2 and st["plans_reused"] == 4 and st["failed"] == 0
    finally:
        B.vdwgb_server_free(sv)


def test_idle_plans_are_evicted_when_the_pool_is_full():
    # a pool that holds one plan of each grid at a time: alternating grids
    # evict the other grid's idle plan, and every request still completes
    g1, g2 = (48, 48, 40), (40, 48, 48)
    foot = max(B.vdwgb_footprint_bytes(g1, B.FP32_MIXED), B.vdwgb_footprint_bytes(g2, B.FP32_MIXED))
    npts = 48 * 48 * 40
    pool = int(1.5 * (foot + 32 * npts + (1 << 20)))
    sv = B.vdwgb_server_new(0, B.FP32_MIXED, pool_bytes=pool, max_batch=1, max_inflight=1)
    try:
        for i in range(4):
            sh = g1 if i % 2 == 0 else g2
            x = np.full(sh, 0.02)
            z = np.zeros(sh)                               # alive until the request is reported
            dn, ds = np.empty(sh), np.empty(sh)
            rid = B.vdwgb_server_submit(sv, 1, sh, np.diag(np.array(sh) * 0.25), x, z, dn, ds)
            e, _ = B.vdwgb_server_wait(sv, rid, 120.0)
            assert np.isfinite(e)
        st = B.vdwgb_server_stats(sv)
        assert st["completed"] == 4 and st["plans_built"] == 4 and st["plans_reused"] == 0
        assert st["pool_used_peak"] <= pool
    finally:
        B.vdwgb_server_free(sv)


@pytest.mark.parametrize("prec", [1, 0])
def test_same_cell_reuse_keeps_the_kpoint_order(prec):
    # one system evaluated repeatedly (an SCF loop) with the functional
    # switching: one plan built, every later request re-plans without the
    # k-point sort and equals a fresh handle bit for bit
    s1 = _requests()[3]
    s2 = inputs.make_system(s1.shape, s1.cell, s1.atoms, 3 - s1.functional)
    alone = {}
    for s in (s1, s2):
        f = B.Functional(s.shape, s.cell, s.functional, prec)
        alone[s.functional] = f.calculate(s.n.numpy(), s.sigma.numpy())
        f.close()
    sv = B.vdwgb_server_new(0, prec, pool_bytes=1 << 30, max_batch=2, max_inflight=1)
    try:
        for k in range(5):
            s = s1 if k % 2 == 0 else s2
            dn, ds = np.empty(s.shape), np.empty(s.shape)
            rid = B.vdwgb_server_submit(sv, s.functional, s.shape, s.cell, s.n.numpy(), s.sigma.numpy(), dn, ds)
            e, _ = B.vdwgb_server_wait(sv, rid, 120.0)
            a = alone[s.functional]
            assert e == a[0] and np.array_equal(dn, a[1]) and np.array_equal(ds, a[2])
        st = B.vdwgb_server_stats(sv)
        assert st["plans_built"] == 1 and st["plans_reused"] == 4
    finally:
        B.vdwgb_server_free(sv)
