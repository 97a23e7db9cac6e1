"""GPU: the bounds-checked build (VDWGB_CHECK_BOUNDS) runs the parity cases
clean.  The checked library is built here (a minute or two) and exercised in
a child process with VDWGB_CHECKED=1: single evaluations on split, unsplit,
odd and triclinic grids in both precisions, a batch in parts, the server,
the allocation-free entry point, the spin-polarised form, two slab ranks, a
caller's kernel table and a 300-point axis, each compared with the oracle
(or one plan) and followed by a clean device status (no access was
skipped)."""
import os
import subprocess
import sys

import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
from paper_1703_06999_gb300 import binding as B, inputs
from oracle import vdw
assert B.LIB_PATH.endswith("libvdwgb_checked.so")
o = vdw.Oracle()
systems = [inputs.small_cubic(0, ngrid=24),
           inputs.make_system((30, 20, 18), np.diag([9.0, 7.0, 6.0]), [(3.0, 1.5, (2.0, 3.0, 1.0))], 2),
           inputs.make_system((15, 21, 35), np.diag([6.0, 8.0, 11.0]), [(4.0, 1.2, (3.0, 4.0, 5.0))], 1),
           inputs.make_system((16, 18, 20), np.array([[7.0, 0, 0], [1.5, 6.5, 0], [-0.8, 1.1, 7.2]]),
                              [(2.0, 1.3, (3.0, 3.0, 3.0))], 1)]
tol = {0: (1e-10, 1e-9), 1: (1e-6, 1e-5)}
for s in systems:
    ref = o.energy_potential(s.n.numpy(), s.sigma.numpy(), s.cell, s.functional)
    for prec in (0, 1):
        f = B.Functional(s.shape, s.cell, s.functional, prec)
        e, dn, ds = f.calculate(s.n.numpy(), s.sigma.numpy())
        f.close()
        et, pt = tol[prec]
        assert abs(e - ref.energy) <= et * max(1.0, abs(ref.energy)), (s.shape, prec, e, ref.energy)
        assert np.max(np.abs(dn - ref.dedn)) <= pt * np.max(np.abs(ref.dedn))
        B.vdwgb_device_status(0)
fs = [B.Functional(s.shape, s.cell, s.functional, 1) for s in systems]
bt = B.vdwgb_batch_new([f.h for f in fs])
hn = [s.n.numpy().copy() for s in systems]
hs = [s.sigma.numpy().copy() for s in systems]
e = B.vdwgb_batch_calculate(bt, hn, hs, [np.empty_like(x) for x in hn], [np.empty_like(x) for x in hn])
B.vdwgb_batch_free(bt)
for f in fs:
    f.close()
sv = B.vdwgb_server_new(0, 1, pool_bytes=1 << 30, max_batch=4, max_inflight=2)
ids, keep = [], []                 # the output arrays live until their requests are done
for s in systems:
    keep.append((np.empty(s.shape), np.empty(s.shape)))
    ids.append(B.vdwgb_server_submit(sv, s.functional, s.shape, s.cell, s.n.numpy(), s.sigma.numpy(), *keep[-1]))
for i in ids:
    B.vdwgb_server_wait(sv, i, 120.0)
B.vdwgb_server_free(sv)
s = systems[0]
n, sg = s.n.cuda(), s.sigma.cuda()
out = torch.empty_like(n)
en = torch.zeros(1, dtype=torch.float64, device="cuda")
B.vdwgb_calculate_noalloc(0, s.functional, s.shape, s.cell, n, sg, out, torch.empty_like(n), en, 0)
torch.cuda.synchronize()
B.vdwgb_device_status(0)
# spin-polarised form, both precisions, against the spin oracle
from oracle import spin as ospin
s = systems[1]
arrs = [x.numpy() for x in inputs.spin_split(s, 0.6, seed=2, empty_down_slab=True)]
sref = ospin.energy_potential_spin(o, *arrs, s.cell, s.functional)
for prec in (0, 1):
    f = B.Functional(s.shape, s.cell, s.functional, prec)
    e, dn, ds = f.calculate_spin(*arrs)
    f.close()
    assert abs(e - sref[0]) <= tol[prec][0] * max(1.0, abs(sref[0])), (prec, e, sref[0])
    B.vdwgb_device_status(0)
# slab decomposition over two virtual ranks: potentials equal one plan
from paper_1703_06999_gb300.slab import LibraryStages
s = systems[0]
st = LibraryStages(0)
P, nxl = 2, s.shape[0] // 2
nb = st.slab_bytes(s.shape, P, 1)
part = nb // P
R = []
for r in range(P):
    a, b, x = st.buffer(nb), st.buffer(nb), st.buffer(nb)
    R.append(dict(h=st.new(s.functional, s.shape, s.cell, P, r, 1, a, b), a=a, b=b, x=x, e=st.energy_buffer(),
                  dn=torch.empty((nxl,) + s.shape[1:], dtype=torch.float64, device="cuda"),
                  ds=torch.empty((nxl,) + s.shape[1:], dtype=torch.float64, device="cuda")))
for r, Rr in enumerate(R):
    st.forward(Rr["h"], n[r * nxl:(r + 1) * nxl].contiguous(), sg[r * nxl:(r + 1) * nxl].contiguous())
    st.pack(Rr["h"], Rr["x"])
for r, Rr in enumerate(R):
    for q, Rq in enumerate(R):
        Rr["b"][q * part:(q + 1) * part].copy_(Rq["x"][r * part:(r + 1) * part])
for Rr in R:
    st.contract(Rr["h"], Rr["e"])
for r, Rr in enumerate(R):
    for q, Rq in enumerate(R):
        Rr["x"][q * part:(q + 1) * part].copy_(Rq["b"][r * part:(r + 1) * part])
for Rr in R:
    st.unpack(Rr["h"], Rr["x"])
    st.inverse(Rr["h"], Rr["dn"], Rr["ds"])
torch.cuda.synchronize()
B.vdwgb_device_status(0)
f = B.Functional(s.shape, s.cell, s.functional, 1)
e1, dn1, ds1 = f.calculate(s.n.numpy(), s.sigma.numpy())
f.close()
assert np.array_equal(torch.cat([Rr["dn"] for Rr in R]).cpu().numpy(), dn1)
for Rr in R:
    st.free(Rr["h"])
# a caller's kernel table and a 300-point axis (several tensor copies per tile)
k = vdw.k_grid(vdw.Params())
gauss = np.tile(np.exp(-0.5 * k * k), (210, 1))
s = systems[2]
f = B.Functional(s.shape, s.cell, s.functional, 1, kernel_k=gauss)
e, dn, ds = f.calculate(s.n.numpy(), s.sigma.numpy())
f.close()
gref = vdw.Oracle(vdw.Params(), phik=gauss).energy_potential(s.n.numpy(), s.sigma.numpy(), s.cell, s.functional)
assert abs(e - gref.energy) <= 1e-6 * max(1.0, abs(gref.energy))
B.vdwgb_device_status(0)
s = inputs.make_system((300, 6, 8), np.diag([60.0, 3.0, 4.0]), [(3.0, 1.5, (20.0, 1.5, 2.0))], 1)
lref = o.energy_potential(s.n.numpy(), s.sigma.numpy(), s.cell, s.functional)
f = B.Functional(s.shape, s.cell, s.functional, 1)
e, dn, ds = f.calculate(s.n.numpy(), s.sigma.numpy())
f.close()
assert abs(e - lref.energy) <= 1e-6 * max(1.0, abs(lref.energy))
B.vdwgb_device_status(0)
print("checked build clean")
'''


def test_checked_build_runs_clean():
    from paper_1703_06999_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, VDWGB_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build clean" in r.stdout
