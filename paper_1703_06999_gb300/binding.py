"""Thin ctypes binding of ``libvdwgb.so`` (C ABI in ``include/vdwgb.h``).

Functions carry the C names and only marshal arguments: every step of the
evaluation runs in the CUDA library.  A missing library raises at load time;
there is no CPU fallback.  torch is used only to hand over device pointers
and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# VDWGB_CHECKED=1 loads the bounds-checked build (build.build(checked=True))
LIB_PATH = os.path.join(HERE, "libvdwgb_checked.so" if os.environ.get("VDWGB_CHECKED") == "1" else "libvdwgb.so")

DF1, DF2 = 1, 2
FP64, FP32_MIXED = 0, 1
INTERP_CUBIC, INTERP_LINEAR = 0, 1
NQ, NPAIR, NK, NR = 20, 210, 1024, 1024

_c_double_p = ctypes.POINTER(ctypes.c_double)
_lib = None

# name: (restype, argtypes)
_SIGS = {
    "vdwgb_new": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "vdwgb_set_unit_cell": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
                            + [ctypes.c_double] * 9),
    "vdwgb_set_interp": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "vdwgb_init_cuda": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "vdwgb_calculate": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 5),
    "vdwgb_calculate_device": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 6),
    "vdwgb_calculate_simple": (ctypes.c_double, [ctypes.c_void_p] + [ctypes.c_void_p] * 4),
    "vdwgb_finalize": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p)]),
    "vdwgb_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "vdwgb_last_error": (ctypes.c_char_p, []),
    "vdwgb_print": (ctypes.c_int, [ctypes.c_void_p]),
    "vdwgb_has_cuda": (ctypes.c_int, []),
    "vdwgb_footprint_bytes": (ctypes.c_size_t, [ctypes.c_int] * 4),
    "vdwgb_launches_per_call": (ctypes.c_int, [ctypes.c_void_p]),
    "vdwgb_device_status": (ctypes.c_int, [ctypes.c_int]),
    "vdwgb_kernel_table": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vdwgb_phi": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vdwgb_table_build_seconds": (ctypes.c_double, [ctypes.c_int]),
    "vdwgb_q0": (ctypes.c_int, [ctypes.c_int] * 4 + [ctypes.c_void_p] * 5),
    "vdwgb_set_autotune": (ctypes.c_int, [ctypes.c_int]),
    "vdwgb_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "vdwgb_set_tiles": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 6),
    "vdwgb_batch_new": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "vdwgb_batch_calculate_device": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 6),
    "vdwgb_batch_free": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p)]),
    "vdwgb_batch_calculate": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 5),
    "vdwgb_batch_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "vdwgb_batch_stage_ms": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "vdwgb_num_stages": (ctypes.c_int, []),
    "vdwgb_batch_launches": (ctypes.c_int, [ctypes.c_void_p]),
    "vdwgb_stage_name": (ctypes.c_char_p, [ctypes.c_int]),
}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("batches", ctypes.c_longlong),
                ("mean_batch", ctypes.c_double), ("pts_per_s", ctypes.c_double),
                ("p50_s", ctypes.c_double), ("p99_s", ctypes.c_double),
                ("pool_bytes", ctypes.c_size_t), ("pool_used_peak", ctypes.c_size_t),
                ("plans_reused", ctypes.c_longlong), ("plans_built", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_SIGS.update({
    "vdwgb_server_new": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "vdwgb_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    "vdwgb_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]),
    "vdwgb_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "vdwgb_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerStats)]),
    "vdwgb_server_free": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p)]),
    "vdwgb_calculate_noalloc": (ctypes.c_int, [ctypes.c_int] * 5 + [ctypes.c_void_p] * 7),
    "vdwgb_set_fused": (ctypes.c_int, [ctypes.c_int]),
    "vdwgb_alu_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "vdwgb_inject_fault": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "vdwgb_slab_bytes": (ctypes.c_size_t, [ctypes.c_int] * 5),
    "vdwgb_slab_new": (ctypes.c_int, [ctypes.c_int] * 4 + [ctypes.c_void_p] + [ctypes.c_int] * 4
                       + [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "vdwgb_slab_forward": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "vdwgb_slab_pack": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "vdwgb_slab_contract": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "vdwgb_slab_unpack": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "vdwgb_slab_inverse": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "vdwgb_slab_free": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p)]),
    "vdwgb_set_kernel_k": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "vdwgb_calculate_spin": (ctypes.c_int, [ctypes.c_void_p] * 10),
    "vdwgb_calculate_spin_device": (ctypes.c_int, [ctypes.c_void_p] * 11),
})


class VdwgbError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = lib().vdwgb_last_error().decode(errors="replace")
        super().__init__("%s failed: %s (%d): %s" % (where, lib().vdwgb_strerror(code).decode(), code, msg))


def lib():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing; build it with __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ck(rc, where):
    if rc != 0:
        raise VdwgbError(rc, where)


def _ptr(a):
    """Address of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


# ---- C-named wrappers ----------------------------------------------------
def vdwgb_new(functional):
    h = ctypes.c_void_p()
    _ck(lib().vdwgb_new(int(functional), ctypes.byref(h)), "vdwgb_new")
    return h


def vdwgb_set_unit_cell(h, shape, cell):
    cell = np.asarray(cell, dtype=np.float64).reshape(9)
    _ck(lib().vdwgb_set_unit_cell(h, int(shape[0]), int(shape[1]), int(shape[2]), *[float(v) for v in cell]),
        "vdwgb_set_unit_cell")


def vdwgb_set_interp(h, interp):
    _ck(lib().vdwgb_set_interp(h, int(interp)), "vdwgb_set_interp")


def vdwgb_init_cuda(h, device=0, precision=FP64):
    _ck(lib().vdwgb_init_cuda(h, int(device), int(precision)), "vdwgb_init_cuda")


def vdwgb_calculate(h, rho, sigma, dedrho, dedsigma):
    """Host arrays (float64, C order); returns the energy."""
    e = np.zeros(1)
    _ck(lib().vdwgb_calculate(h, _ptr(rho), _ptr(sigma), _ptr(dedrho), _ptr(dedsigma), e.ctypes.data),
        "vdwgb_calculate")
    return float(e[0])


def vdwgb_calculate_device(h, rho, sigma, dedrho, dedsigma, energy, stream=0):
    """Device tensors (float64, contiguous); ``stream`` is a raw cudaStream_t."""
    _ck(lib().vdwgb_calculate_device(h, _ptr(rho), _ptr(sigma), _ptr(dedrho), _ptr(dedsigma), _ptr(energy),
                                     ctypes.c_void_p(int(stream))), "vdwgb_calculate_device")


def vdwgb_calculate_spin(h, rho_up, rho_dn, sigma_upup, sigma_dndn, dedrho_up, dedrho_dn, dedsigma_upup,
                         dedsigma_dndn):
    """Spin-polarised form, host arrays (float64, C order); returns the energy."""
    e = np.zeros(1)
    _ck(lib().vdwgb_calculate_spin(h, _ptr(rho_up), _ptr(rho_dn), _ptr(sigma_upup), _ptr(sigma_dndn),
                                   _ptr(dedrho_up), _ptr(dedrho_dn), _ptr(dedsigma_upup), _ptr(dedsigma_dndn),
                                   e.ctypes.data), "vdwgb_calculate_spin")
    return float(e[0])


def vdwgb_calculate_spin_device(h, rho_up, rho_dn, sigma_upup, sigma_dndn, dedrho_up, dedrho_dn, dedsigma_upup,
                                dedsigma_dndn, energy, stream=0):
    """Spin-polarised form, device tensors (float64, contiguous); ``stream`` a raw cudaStream_t."""
    _ck(lib().vdwgb_calculate_spin_device(h, _ptr(rho_up), _ptr(rho_dn), _ptr(sigma_upup), _ptr(sigma_dndn),
                                          _ptr(dedrho_up), _ptr(dedrho_dn), _ptr(dedsigma_upup),
                                          _ptr(dedsigma_dndn), _ptr(energy), ctypes.c_void_p(int(stream))),
        "vdwgb_calculate_spin_device")


def vdwgb_set_kernel_k(h, phik):
    """A caller's kernel table phi_ab(k_j) (210 x 1024 float64, pairs a <= b
    row-major) before init; None restores the vdW-DF table."""
    if phik is None:
        _ck(lib().vdwgb_set_kernel_k(h, None), "vdwgb_set_kernel_k")
        return
    a = np.ascontiguousarray(phik, dtype=np.float64)
    if a.size != 210 * 1024:
        raise ValueError("kernel table must hold 210 x 1024 values")
    _ck(lib().vdwgb_set_kernel_k(h, a.ctypes.data), "vdwgb_set_kernel_k")


def vdwgb_set_fused(enable):
    """Plane kernel on or off for handles initialised afterwards."""
    _ck(lib().vdwgb_set_fused(int(bool(enable))), "vdwgb_set_fused")


def vdwgb_calculate_noalloc(device, functional, shape, cell, rho, sigma, dedrho, dedsigma, energy, stream=0):
    """Handle-free evaluation without device allocation (device tensors,
    float64, contiguous; FP32-mixed, cubic).  The kernel table of ``device``
    must be resident (``vdwgb_kernel_table``)."""
    cell = np.ascontiguousarray(np.asarray(cell, dtype=np.float64).reshape(9))
    _ck(lib().vdwgb_calculate_noalloc(int(device), int(functional), int(shape[0]), int(shape[1]), int(shape[2]),
                                      cell.ctypes.data, _ptr(rho), _ptr(sigma), _ptr(dedrho), _ptr(dedsigma),
                                      _ptr(energy), ctypes.c_void_p(int(stream))), "vdwgb_calculate_noalloc")


def vdwgb_calculate_simple(h, rho, sigma, dedrho, dedsigma):
    return float(lib().vdwgb_calculate_simple(h, _ptr(rho), _ptr(sigma), _ptr(dedrho), _ptr(dedsigma)))


def vdwgb_finalize(h):
    _ck(lib().vdwgb_finalize(ctypes.byref(h)), "vdwgb_finalize")


def vdwgb_strerror(code):
    return lib().vdwgb_strerror(int(code)).decode()


def vdwgb_last_error():
    return lib().vdwgb_last_error().decode(errors="replace")


def vdwgb_print(h):
    _ck(lib().vdwgb_print(h), "vdwgb_print")


def vdwgb_has_cuda():
    return bool(lib().vdwgb_has_cuda())


def vdwgb_footprint_bytes(shape, precision):
    return int(lib().vdwgb_footprint_bytes(int(shape[0]), int(shape[1]), int(shape[2]), int(precision)))


def vdwgb_device_status(device=0):
    _ck(lib().vdwgb_device_status(int(device)), "vdwgb_device_status")


def vdwgb_slab_bytes(shape, P, precision):
    nx, ny, nz = (int(v) for v in shape)
    return int(lib().vdwgb_slab_bytes(nx, ny, nz, int(P), int(precision)))


def vdwgb_slab_new(functional, shape, cell, P, rank, device, precision, aspec, bspec):
    nx, ny, nz = (int(v) for v in shape)
    c = np.ascontiguousarray(np.asarray(cell, dtype=np.float64).reshape(9))
    h = ctypes.c_void_p()
    _ck(lib().vdwgb_slab_new(int(functional), nx, ny, nz, c.ctypes.data, int(P), int(rank), int(device),
                             int(precision), _ptr(aspec), _ptr(bspec), ctypes.byref(h)), "vdwgb_slab_new")
    return h


def vdwgb_slab_forward(s, rho, sigma, stream=0):
    _ck(lib().vdwgb_slab_forward(s, _ptr(rho), _ptr(sigma), stream), "vdwgb_slab_forward")


def vdwgb_slab_pack(s, send, stream=0):
    _ck(lib().vdwgb_slab_pack(s, _ptr(send), stream), "vdwgb_slab_pack")


def vdwgb_slab_contract(s, energy, stream=0):
    _ck(lib().vdwgb_slab_contract(s, _ptr(energy), stream), "vdwgb_slab_contract")


def vdwgb_slab_unpack(s, recv, stream=0):
    _ck(lib().vdwgb_slab_unpack(s, _ptr(recv), stream), "vdwgb_slab_unpack")


def vdwgb_slab_inverse(s, dedrho, dedsigma, stream=0):
    _ck(lib().vdwgb_slab_inverse(s, _ptr(dedrho), _ptr(dedsigma), stream), "vdwgb_slab_inverse")


def vdwgb_slab_free(s):
    _ck(lib().vdwgb_slab_free(ctypes.byref(s)), "vdwgb_slab_free")


FAULT_NONE, FAULT_ALLOC, FAULT_WAIT = 0, 1, 2


def vdwgb_inject_fault(kind, count=1):
    """Arm a fault for tests: FAULT_ALLOC (next `count` device allocations
    fail: ENOMEM), FAULT_WAIT (next `count` status checks find the device's
    timeout flag set: ETIMEDOUT), FAULT_NONE (disarm)."""
    _ck(lib().vdwgb_inject_fault(int(kind), int(count)), "vdwgb_inject_fault")


def vdwgb_alu_peak(kind, device=0):
    """Measured GFLOP/s of the CUDA cores: kind 0 FP32, 1 FP32x2, 2 FP64."""
    g = ctypes.c_double(0.0)
    _ck(lib().vdwgb_alu_peak(int(device), int(kind), ctypes.byref(g)), "vdwgb_alu_peak")
    return g.value


def vdwgb_batch_launches(b):
    return int(lib().vdwgb_batch_launches(b))


def vdwgb_launches_per_call(h):
    return int(lib().vdwgb_launches_per_call(h))


def vdwgb_kernel_table(device=0):
    phik = np.zeros((NPAIR, NK))
    phir = np.zeros((NPAIR, NR + 1))
    q = np.zeros(NQ)
    _ck(lib().vdwgb_kernel_table(int(device), phik.ctypes.data, phir.ctypes.data, q.ctypes.data),
        "vdwgb_kernel_table")
    return phik, phir, q


def vdwgb_phi(d1, d2, device=0):
    d1 = np.ascontiguousarray(d1, dtype=np.float64).ravel()
    d2 = np.ascontiguousarray(d2, dtype=np.float64).ravel()
    out = np.zeros(d1.size)
    _ck(lib().vdwgb_phi(int(device), d1.size, d1.ctypes.data, d2.ctypes.data, out.ctypes.data), "vdwgb_phi")
    return out


def vdwgb_q0(n, sigma, functional=DF1, precision=FP64, device=0):
    """(q0, dq0/dn, dq0/dsigma) as the given precision form computes them."""
    n = np.ascontiguousarray(n, dtype=np.float64).ravel()
    sigma = np.ascontiguousarray(sigma, dtype=np.float64).ravel()
    q0, dn, ds = np.zeros(n.size), np.zeros(n.size), np.zeros(n.size)
    _ck(lib().vdwgb_q0(int(device), int(precision), int(functional), n.size, n.ctypes.data, sigma.ctypes.data,
                       q0.ctypes.data, dn.ctypes.data, ds.ctypes.data), "vdwgb_q0")
    return q0, dn, ds


def vdwgb_set_autotune(enable):
    _ck(lib().vdwgb_set_autotune(int(bool(enable))), "vdwgb_set_autotune")


def vdwgb_set_tiles(h, lz, lzi, wy, wx, nby, nbx):
    _ck(lib().vdwgb_set_tiles(h, int(lz), int(lzi), int(wy), int(wx), int(nby), int(nbx)), "vdwgb_set_tiles")


def vdwgb_plan_info(h):
    info = np.zeros(9, dtype=np.int32)
    _ck(lib().vdwgb_plan_info(h, info.ctypes.data), "vdwgb_plan_info")
    keys = ["LZ", "LZi", "Wy", "Wx", "nbuf_yx", "chunks", "launches", "autotuned", "cluster"]
    return {k: int(v) for k, v in zip(keys, info)}


def vdwgb_table_build_seconds(device=0):
    return float(lib().vdwgb_table_build_seconds(int(device)))


def vdwgb_batch_new(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    b = ctypes.c_void_p()
    _ck(lib().vdwgb_batch_new(arr, len(handles), ctypes.byref(b)), "vdwgb_batch_new")
    return b


def vdwgb_batch_calculate_device(b, rhos, sigmas, dedrhos, dedsigmas, energies, stream=0):
    n = len(rhos)
    P = ctypes.c_void_p * n
    _ck(lib().vdwgb_batch_calculate_device(b, P(*[_ptr(t) for t in rhos]), P(*[_ptr(t) for t in sigmas]),
                                           P(*[_ptr(t) for t in dedrhos]), P(*[_ptr(t) for t in dedsigmas]),
                                           _ptr(energies), ctypes.c_void_p(int(stream))),
        "vdwgb_batch_calculate_device")


def vdwgb_batch_calculate(b, rhos, sigmas, dedrhos, dedsigmas):
    """Host arrays (numpy float64, C order, pinned or pageable); returns energies."""
    n = len(rhos)
    P = ctypes.c_void_p * n
    e = np.zeros(n)
    _ck(lib().vdwgb_batch_calculate(b, P(*[_ptr(t) for t in rhos]), P(*[_ptr(t) for t in sigmas]),
                                    P(*[_ptr(t) for t in dedrhos]), P(*[_ptr(t) for t in dedsigmas]),
                                    e.ctypes.data), "vdwgb_batch_calculate")
    return e


def vdwgb_batch_set_timing(b, enable):
    _ck(lib().vdwgb_batch_set_timing(b, int(bool(enable))), "vdwgb_batch_set_timing")


def vdwgb_num_stages():
    return int(lib().vdwgb_num_stages())


def vdwgb_stage_name(i):
    return lib().vdwgb_stage_name(int(i)).decode()


def vdwgb_batch_stage_ms(b):
    """(per-stage summed milliseconds, number of timed calls)."""
    ms = np.zeros(vdwgb_num_stages())
    nc = ctypes.c_int(0)
    _ck(lib().vdwgb_batch_stage_ms(b, ms.ctypes.data, ctypes.byref(nc)), "vdwgb_batch_stage_ms")
    return ms, int(nc.value)


def vdwgb_batch_free(b):
    _ck(lib().vdwgb_batch_free(ctypes.byref(b)), "vdwgb_batch_free")


def vdwgb_server_new(device=0, precision=FP32_MIXED, pool_bytes=8 << 30, max_batch=16, max_inflight=2):
    sv = ctypes.c_void_p()
    _ck(lib().vdwgb_server_new(int(device), int(precision), int(pool_bytes), int(max_batch), int(max_inflight),
                               ctypes.byref(sv)), "vdwgb_server_new")
    return sv


def vdwgb_server_submit(sv, functional, shape, cell, rho, sigma, dedrho, dedsigma):
    """Host arrays (numpy float64, C order) owned by the caller until done; returns the id."""
    cell = np.ascontiguousarray(np.asarray(cell, dtype=np.float64).reshape(9))
    rid = ctypes.c_longlong()
    _ck(lib().vdwgb_server_submit(sv, int(functional), int(shape[0]), int(shape[1]), int(shape[2]),
                                  cell.ctypes.data, _ptr(rho), _ptr(sigma), _ptr(dedrho), _ptr(dedsigma),
                                  ctypes.byref(rid)), "vdwgb_server_submit")
    return int(rid.value)


def vdwgb_server_poll(sv, rid):
    """None if pending, else (energy, latency_s)."""
    e, t = ctypes.c_double(), ctypes.c_double()
    rc = lib().vdwgb_server_poll(sv, int(rid), ctypes.byref(e), ctypes.byref(t))
    if rc == 0:
        return None
    if rc < 0:
        raise VdwgbError(rc, "vdwgb_server_poll")
    return e.value, t.value


def vdwgb_server_wait(sv, rid, timeout_s=60.0):
    e, t = ctypes.c_double(), ctypes.c_double()
    rc = lib().vdwgb_server_wait(sv, int(rid), float(timeout_s), ctypes.byref(e), ctypes.byref(t))
    if rc < 0:
        raise VdwgbError(rc, "vdwgb_server_wait")
    return e.value, t.value


def vdwgb_server_stats(sv):
    st = ServerStats()
    _ck(lib().vdwgb_server_stats(sv, ctypes.byref(st)), "vdwgb_server_stats")
    return st.as_dict()


def vdwgb_server_free(sv):
    _ck(lib().vdwgb_server_free(ctypes.byref(sv)), "vdwgb_server_free")


# ---- convenience ------------------------------------------------------------
class Functional:
    """One initialised handle: ``Functional(shape, cell, functional, precision)``."""

    def __init__(self, shape, cell, functional=DF1, precision=FP64, device=0, interp=INTERP_CUBIC, kernel_k=None):
        self.shape = tuple(int(v) for v in shape)
        self.h = vdwgb_new(functional)
        try:
            vdwgb_set_unit_cell(self.h, self.shape, cell)
            vdwgb_set_interp(self.h, interp)
            if kernel_k is not None:
                vdwgb_set_kernel_k(self.h, kernel_k)
            vdwgb_init_cuda(self.h, device, precision)
        except Exception:
            vdwgb_finalize(self.h)
            raise

    def calculate(self, rho, sigma):
        """Host float64 arrays in; (energy, dedrho, dedsigma) out."""
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        dn = np.empty_like(rho)
        ds = np.empty_like(rho)
        e = vdwgb_calculate(self.h, rho, sigma, dn, ds)
        return e, dn, ds

    def calculate_device(self, rho, sigma, dedrho, dedsigma, energy, stream=0):
        vdwgb_calculate_device(self.h, rho, sigma, dedrho, dedsigma, energy, stream)

    def calculate_spin(self, rho_up, rho_dn, sigma_upup, sigma_dndn):
        """Spin-polarised form, host float64 arrays in; (energy, (dE/dn_up,
        dE/dn_dn), (dE/dsigma_upup, dE/dsigma_dndn)) out."""
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (rho_up, rho_dn, sigma_upup, sigma_dndn)]
        o = [np.empty_like(a[0]) for _ in range(4)]
        e = vdwgb_calculate_spin(self.h, *a, *o)
        return e, (o[0], o[1]), (o[2], o[3])

    def close(self):
        if self.h is not None and self.h.value:
            vdwgb_finalize(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
