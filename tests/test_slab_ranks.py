"""The slab driver's exchanges (two all-to-alls of equal parts and the sum
of the energy parts) over two gloo ranks on CPU.  A numpy stand-in of the
library's slab stages, built from the oracle's pieces, computes each rank's
share on its x-slab / ky-slab with the same buffer layouts as the library
([xl][y][kz][a] spectrum, [d][xl][run] send order); the ranks' gathered
result must equal the oracle on the whole grid."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class NumpyStages:
    """The slab stages of one rank on CPU tensors, FP64 (16-byte complex)."""

    def __init__(self, oracle):
        self.o = oracle
        self.M = oracle.p.M

    def slab_bytes(self, shape, P, precision):
        nx, ny, nz = shape
        if nx % P or ny % P:
            return 0
        return (nx // P) * ny * (nz // 2 + 1) * self.M * 16

    def buffer(self, nbytes):
        return torch.zeros(nbytes, dtype=torch.uint8)

    def energy_buffer(self):
        return torch.zeros(1, dtype=torch.float64)

    def new(self, functional, shape, cell, P, rank, precision, aspec, bspec):
        return dict(functional=functional, shape=tuple(shape), cell=np.asarray(cell, dtype=np.float64), P=P,
                    rank=rank, aspec=aspec, bspec=bspec)

    def _spec(self, buf, dims):
        return buf.view(torch.complex128).numpy().reshape(dims + (self.M,))

    def forward(self, h, rho, sigma):
        nx, ny, nz = h["shape"]
        n, s = rho.numpy(), sigma.numpy()
        theta, q0, dq_dn, dq_ds, pa, dpa, live = self.o.theta(n, s, h["functional"])
        h["pot"] = (n, dq_dn, dq_ds, pa, dpa, live)
        th = np.fft.fft(np.fft.rfft(theta, axis=3), axis=2)          # (M, nxl, ny, nzh)
        self._spec(h["aspec"], (nx // h["P"], ny, nz // 2 + 1))[...] = np.moveaxis(th, 0, -1)

    def pack(self, h, send):
        nx, ny, nz = h["shape"]
        P = h["P"]
        a = self._spec(h["aspec"], (nx // P, P, ny // P, nz // 2 + 1))
        self._spec(send, (P, nx // P, ny // P, nz // 2 + 1))[...] = a.transpose(1, 0, 2, 3, 4)

    def contract(self, h, energy):
        nx, ny, nz = h["shape"]
        P, r = h["P"], h["rank"]
        nyl, nzh = ny // P, nz // 2 + 1
        b = self._spec(h["bspec"], (nx, nyl, nzh))
        th = np.fft.fft(np.moveaxis(b, -1, 0), axis=1)                # theta_a(k) on the ky-slab
        from oracle import vdw
        kabs = vdw.kabs_grid((nx, ny, nz), h["cell"])[:, r * nyl:(r + 1) * nyl, :nzh]
        phi = self.o.kernel_matrix(kabs)
        F = np.einsum("abxyz,bxyz->axyz", phi, th)
        w = np.full(nzh, 2.0)
        w[0] = 1.0
        if nz % 2 == 0:
            w[-1] = 1.0
        N = float(nx * ny * nz)
        omega = vdw.cell_volume(h["cell"])
        energy[0] = 0.5 * omega / (N * N) * float(np.sum(w * np.real(np.conj(th) * F)))
        b[...] = np.moveaxis(np.fft.ifft(F, axis=1), 0, -1)

    def unpack(self, h, recv):
        nx, ny, nz = h["shape"]
        P = h["P"]
        src = self._spec(recv, (P, nx // P, ny // P, nz // 2 + 1))
        self._spec(h["aspec"], (nx // P, P, ny // P, nz // 2 + 1))[...] = src.transpose(1, 0, 2, 3, 4)

    def inverse(self, h, dedrho, dedsigma):
        nx, ny, nz = h["shape"]
        a = self._spec(h["aspec"], (nx // h["P"], ny, nz // 2 + 1))
        F = np.fft.irfft(np.fft.ifft(np.moveaxis(a, -1, 0), axis=2), n=nz, axis=3)
        n, dq_dn, dq_ds, pa, dpa, live = h["pot"]
        dn = np.sum(F * (pa + n * dpa * dq_dn), axis=0)
        ds = n * np.sum(F * dpa, axis=0) * dq_ds
        dedrho.numpy()[...] = np.where(live, dn, 0.0)
        dedsigma.numpy()[...] = np.where(live, ds, 0.0)

    def status(self):
        pass

    def free(self, h):
        h.clear()


def _system():
    from paper_1703_06999_gb300 import inputs
    g = np.random.default_rng(4)
    shape = (12, 10, 14)
    L = np.array(shape) * 0.45
    cell = np.array([[L[0], 0, 0], [0.6, L[1], 0], [-0.3, 0.5, L[2]]])
    atoms = [(float(g.uniform(1, 6)), float(g.uniform(1, 2.5)), tuple(g.uniform(0, 1, 3) @ cell))
             for _ in range(3)]
    return inputs.make_system(shape, cell, atoms, 2)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import vdw
        from paper_1703_06999_gb300.slab import SlabEvaluator
        s = _system()
        nxl = s.shape[0] // world
        ev = SlabEvaluator(s.shape, s.cell, s.functional, 0, stages=NumpyStages(vdw.Oracle(vdw.Params())))
        assert ev.P == world and ev.rank == rank
        sl = slice(rank * nxl, (rank + 1) * nxl)
        dn = torch.empty((nxl,) + s.shape[1:], dtype=torch.float64)
        ds = torch.empty_like(dn)
        e = ev.calculate(s.n[sl].contiguous(), s.sigma[sl].contiguous(), dn, ds)
        ev.close()
        q.put((rank, e, dn.numpy().copy(), ds.numpy().copy()))
        dist.barrier()
    except BaseException as ex:          # reported to the parent instead of a silent hang
        q.put((rank, repr(ex), None, None))
        raise
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_oracle_on_whole_grid(oracle_default):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(2)], key=lambda t: t[0])
    assert all(r[2] is not None for r in res), res
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = _system()
    ref = oracle_default.energy_potential(s.n.numpy(), s.sigma.numpy(), s.cell, s.functional)
    assert res[0][1] == res[1][1]                                 # every rank holds the summed energy
    assert abs(res[0][1] - ref.energy) <= 1e-12 * abs(ref.energy)
    dn = np.concatenate([r[2] for r in res])
    ds = np.concatenate([r[3] for r in res])
    assert np.max(np.abs(dn - ref.dedn)) <= 1e-11 * np.max(np.abs(ref.dedn))
    assert np.max(np.abs(ds - ref.dedsigma)) <= 1e-11 * np.max(np.abs(ref.dedsigma))


def test_single_rank_without_process_group(oracle_default):
    from paper_1703_06999_gb300.slab import SlabEvaluator
    s = _system()
    ev = SlabEvaluator(s.shape, s.cell, s.functional, 0, stages=NumpyStages(oracle_default))
    assert ev.P == 1
    dn = torch.empty(s.shape, dtype=torch.float64)
    ds = torch.empty_like(dn)
    e = ev.calculate(s.n, s.sigma, dn, ds)
    ev.close()
    ref = oracle_default.energy_potential(s.n.numpy(), s.sigma.numpy(), s.cell, s.functional)
    assert abs(e - ref.energy) <= 1e-12 * abs(ref.energy)
    assert np.max(np.abs(dn.numpy() - ref.dedn)) <= 1e-11 * np.max(np.abs(ref.dedn))


def test_grid_not_divisible_is_rejected(oracle_default):
    from paper_1703_06999_gb300.slab import SlabEvaluator

    class Three(NumpyStages):
        def slab_bytes(self, shape, P, precision):
            return super().slab_bytes(shape, 3, precision)
    with pytest.raises(ValueError):
        SlabEvaluator((12, 10, 14), np.eye(3) * 6, 1, 0, stages=Three(oracle_default))
