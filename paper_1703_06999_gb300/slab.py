"""Slab decomposition of one system over the ranks of a torch.distributed
group (one GPU per rank): the paper's parallel layout (Sec. 3,
parallelisation: slabs of x-planes, the spectrum distributed over y) with
the library's slab stages (``vdwgb_slab_*`` in ``include/vdwgb.h``) and two
all-to-all exchanges of equal parts plus one all-reduce of the energy.

Each rank passes its x-slab (``nx/P`` planes) of rho and sigma and receives
the same slab of dE/drho and dE/dsigma and the total energy.  Argument
marshalling and the collectives only: every arithmetic step runs in the
library's kernels.
"""
from __future__ import annotations

from . import binding as B


class LibraryStages:
    """The CUDA library's slab stages on the current CUDA device and stream."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)

    def slab_bytes(self, shape, P, precision):
        return B.vdwgb_slab_bytes(shape, P, precision)

    def buffer(self, nbytes):
        return self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.device)

    def energy_buffer(self):
        return self.torch.zeros(1, dtype=self.torch.float64, device=self.device)

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def new(self, functional, shape, cell, P, rank, precision, aspec, bspec):
        return B.vdwgb_slab_new(functional, shape, cell, P, rank, self.device.index, precision, aspec, bspec)

    def forward(self, h, rho, sigma):
        B.vdwgb_slab_forward(h, rho, sigma, self._stream())

    def pack(self, h, send):
        B.vdwgb_slab_pack(h, send, self._stream())

    def contract(self, h, energy):
        B.vdwgb_slab_contract(h, energy, self._stream())

    def unpack(self, h, recv):
        B.vdwgb_slab_unpack(h, recv, self._stream())

    def inverse(self, h, dedrho, dedsigma):
        B.vdwgb_slab_inverse(h, dedrho, dedsigma, self._stream())

    def status(self):
        B.vdwgb_device_status(self.device.index)

    def free(self, h):
        B.vdwgb_slab_free(h)


class SlabEvaluator:
    """This rank's share of a slab-decomposed evaluation of one system of
    grid ``shape`` (nx and ny multiples of the group size P).

    ``calculate(rho, sigma, dedrho, dedsigma)`` takes this rank's x-slab
    (``(nx/P, ny, nz)`` arrays of the stages' kind: CUDA float64 tensors for
    the library) and returns the total energy (Hartree); dedrho and dedsigma
    receive the slab's potentials.  ``stages`` defaults to the CUDA library;
    anything with the same methods can stand in (the tests run the exchange
    logic on CPU ranks that way)."""

    def __init__(self, shape, cell, functional=B.DF1, precision=B.FP32_MIXED, group=None, stages=None):
        import torch.distributed as dist
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.group = group
        self.P = self.dist.get_world_size(group) if self.dist else 1
        self.rank = self.dist.get_rank(group) if self.dist else 0
        self.stages = stages if stages is not None else LibraryStages()
        self.shape = tuple(int(v) for v in shape)
        nbytes = self.stages.slab_bytes(self.shape, self.P, precision)
        if nbytes == 0:
            raise ValueError("grid %s: nx and ny must be multiples of %d ranks" % (self.shape, self.P))
        # x-slab spectrum, ky-slab spectrum (the forward exchange's receive
        # buffer), exchange buffer (forward send, inverse receive)
        self.aspec = self.stages.buffer(nbytes)
        self.bspec = self.stages.buffer(nbytes)
        self.xbuf = self.stages.buffer(nbytes)
        self.h = self.stages.new(functional, self.shape, cell, self.P, self.rank, precision, self.aspec, self.bspec)

    def _all_to_all(self, out, inp):
        if self.P == 1:
            out.copy_(inp)
        else:
            self.dist.all_to_all_single(out, inp, group=self.group)

    def calculate(self, rho, sigma, dedrho, dedsigma):
        st = self.stages
        energy = st.energy_buffer()
        st.forward(self.h, rho, sigma)
        st.pack(self.h, self.xbuf)
        self._all_to_all(self.bspec, self.xbuf)     # x-slabs -> ky-slabs
        st.contract(self.h, energy)
        self._all_to_all(self.xbuf, self.bspec)     # ky-slabs -> x-slabs
        st.unpack(self.h, self.xbuf)
        st.inverse(self.h, dedrho, dedsigma)
        if self.P > 1:
            self.dist.all_reduce(energy, group=self.group)
        e = float(energy[0])
        st.status()
        return e

    def close(self):
        if self.h is not None:
            self.stages.free(self.h)
            self.h = None
