"""Seeded synthetic densities for the vdW-DF nonlocal-correlation path.

This module holds no arithmetic of the vdW-DF method: it only makes inputs
(a density n on a periodic grid and sigma = |grad n|^2) with the shapes and
structure of the paper's workloads.  Both the CUDA path and the FP64 oracle
are fed from here; nothing here depends on either.

Density model: a floor plus periodic atom-like exponentials
    n(r) = floor + sum_a sum_R Z_a zeta_a^3 / (8 pi) exp(-zeta_a |r - R_a - R|)
(each term integrates to Z_a electrons).  Periodic images R are summed while
zeta_a |r - R_a - R| <= 30 can occur (exp(-30) ~ 1e-13 of the peak, below the
floor).  sigma is |grad n|^2 from a spectral
gradient with the Nyquist component of each axis zeroed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np
import torch

Atom = Tuple[float, float, Tuple[float, float, float]]   # (Z, zeta, centre)


@dataclass
class System:
    """One synthetic evaluation: grid shape, cell (rows = lattice vectors,
    bohr), functional id (1 = vdW-DF1, 2 = vdW-DF2), n and sigma (float64)."""
    shape: Tuple[int, int, int]
    cell: np.ndarray
    functional: int
    n: torch.Tensor
    sigma: torch.Tensor
    atoms: List[Atom] = field(default_factory=list)
    name: str = ""

    @property
    def npts(self) -> int:
        return int(self.shape[0] * self.shape[1] * self.shape[2])


def _grid_coords(shape, cell, device):
    cell_t = torch.as_tensor(np.asarray(cell, dtype=np.float64), device=device)
    fr = [torch.arange(s, dtype=torch.float64, device=device) / s for s in shape]
    fx, fy, fz = torch.meshgrid(*fr, indexing="ij")
    frac = torch.stack([fx, fy, fz], dim=-1)            # (nx, ny, nz, 3)
    return frac @ cell_t                                 # cartesian


def density(shape, cell, atoms: Sequence[Atom], floor: float = 1e-10,
            device="cpu", cutoff: float = 30.0) -> torch.Tensor:
    """n(r) on the grid (float64, [nx][ny][nz], z contiguous).  Every periodic
    image of an atom that can come within zeta |r - R| <= cutoff of the cell
    contributes; the images are evaluated in groups (one pass over the grid
    per group) to keep the number of device operations small.  On a GPU the
    distances, exponentials and the sum over a group's images are evaluated
    in FP32 (the GPU's FP64 rate is a small fraction of its FP32 rate; the
    density then differs from an FP64 evaluation by about 1e-5 relative), and
    the groups are summed in FP64."""
    cell = np.asarray(cell, dtype=np.float64)
    r = _grid_coords(shape, cell, device).reshape(-1, 3)
    npts = r.shape[0]
    # shortest distance between opposite faces, for the image range
    vol = abs(np.linalg.det(cell))
    heights = [vol / np.linalg.norm(np.cross(cell[(i + 1) % 3], cell[(i + 2) % 3])) for i in range(3)]
    mid = 0.5 * cell.sum(axis=0)
    half_diag = 0.5 * max(np.linalg.norm(cell[0] * sx + cell[1] * sy + cell[2] * sz)
                          for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1))
    centres, zetas, prefs = [], [], []
    for Z, zeta, centre in atoms:
        reach = cutoff / zeta
        nimg = [int(math.ceil(reach / h)) + 1 for h in heights]
        pref = Z * zeta ** 3 / (8.0 * math.pi)
        ijk = np.stack(np.meshgrid(*[np.arange(-m, m + 1) for m in nimg], indexing="ij"), axis=-1).reshape(-1, 3)
        shifts = np.asarray(centre, dtype=np.float64) + ijk @ cell
        keep = (np.linalg.norm(shifts - mid, axis=1) - half_diag) * zeta <= cutoff   # images that reach the cell
        centres.append(shifts[keep])
        zetas.append(np.full(int(keep.sum()), zeta))
        prefs.append(np.full(int(keep.sum()), pref))
    n = torch.full((npts,), float(floor), dtype=torch.float64, device=device)
    centres = np.concatenate(centres) if centres else np.zeros((0, 3))
    if len(centres):
        gpu = torch.device(device).type == "cuda"
        fdt = torch.float32 if gpu else torch.float64
        c = torch.as_tensor(centres, dtype=fdt, device=device)
        zt = torch.as_tensor(np.concatenate(zetas), dtype=fdt, device=device)
        pf = torch.as_tensor(np.concatenate(prefs), dtype=fdt, device=device)
        rx, ry, rz = (r[:, q].to(fdt).contiguous() for q in range(3))
        group = max(1, (1 << 26) // max(npts, 1))          # about 256 MB per intermediate
        for g0 in range(0, len(centres), group):
            g1 = min(len(centres), g0 + group)
            d2 = rx[None, :] - c[g0:g1, 0:1]
            d2.square_()
            t = ry[None, :] - c[g0:g1, 1:2]
            d2.addcmul_(t, t)
            t = rz[None, :] - c[g0:g1, 2:3]
            d2.addcmul_(t, t)
            d2.sqrt_().mul_(-zt[g0:g1, None]).exp_()       # exp(-zeta |r - R|) per image and point
            n += (pf[None, g0:g1] @ d2).reshape(-1).to(torch.float64)
    return n.reshape(tuple(shape))


def spectral_sigma(n: torch.Tensor, cell) -> torch.Tensor:
    """sigma = |grad n|^2 with the gradient taken spectrally (Nyquist zeroed)."""
    shape = n.shape
    dev = n.device
    cell = np.asarray(cell, dtype=np.float64)
    B = torch.as_tensor(2.0 * np.pi * np.linalg.inv(cell).T, device=dev)   # rows b_j
    nk = torch.fft.fftn(n)
    ms = []
    for s in shape:
        m = torch.fft.fftfreq(s, 1.0 / s, dtype=torch.float64, device=dev)
        if s % 2 == 0:
            m[s // 2] = 0.0
        ms.append(m)
    mx, my, mz = torch.meshgrid(*ms, indexing="ij")
    sig = torch.zeros(shape, dtype=torch.float64, device=dev)
    for c in range(3):
        kc = mx * B[0, c] + my * B[1, c] + mz * B[2, c]
        g = torch.fft.ifftn(1j * kc * nk).real
        sig += g * g
    return sig


def make_system(shape, cell, atoms, functional=1, floor=1e-10, device="cpu", name="") -> System:
    n = density(shape, cell, atoms, floor, device)
    s = spectral_sigma(n, cell)
    return System(tuple(int(v) for v in shape), np.asarray(cell, dtype=np.float64),
                  int(functional), n, s, list(atoms), name)


def spin_split(system: System, amplitude: float = 0.6, seed: int = 0, empty_down_slab: bool = False):
    """Spin densities of a system: n_up = n (1 + zeta) / 2, n_dn = n (1 - zeta) / 2
    with a smooth periodic polarisation zeta(r) = amplitude sin(2 pi (u . f1))
    cos(2 pi (u . f2)) (u the fractional coordinates, f1 and f2 small integer
    vectors drawn from ``seed``), and sigma_ss = |grad n_s|^2 spectrally.
    ``empty_down_slab`` makes the first quarter of the x planes fully
    polarised (n_dn = 0 there).  Returns (n_up, n_dn, sigma_upup, sigma_dndn),
    float64 tensors on the system's device."""
    g = _rng(seed)
    n = system.n
    dev = n.device
    fr = [torch.arange(k, dtype=torch.float64, device=dev) / k for k in system.shape]
    u = torch.stack(torch.meshgrid(*fr, indexing="ij"), dim=-1)
    f1 = torch.as_tensor(g.integers(-2, 3, 3), dtype=torch.float64, device=dev)
    f2 = torch.as_tensor(g.integers(-2, 3, 3), dtype=torch.float64, device=dev)
    f1[0] = 1.0
    zeta = amplitude * torch.sin(2 * np.pi * (u @ f1)) * torch.cos(2 * np.pi * (u @ f2))
    if empty_down_slab:
        zeta[: max(1, system.shape[0] // 4)] = 1.0
    nu = n * (1 + zeta) / 2
    nd = n * (1 - zeta) / 2
    return nu, nd, spectral_sigma(nu, system.cell), spectral_sigma(nd, system.cell)


# ---------------------------------------------------------------------------
# Workloads (sizes and structure of the paper's use cases, all synthetic).
# ---------------------------------------------------------------------------
def _rng(seed):
    return np.random.default_rng(seed)


def small_cubic(seed=0, ngrid=24, L=10.0, natoms=4, functional=1, device="cpu") -> System:
    """24^3 grid in a cubic 10 bohr cell, 4 exponentials with Z in [1, 8],
    zeta in [1, 3] and uniform centres, floor 1e-10."""
    g = _rng(seed)
    atoms = [(float(g.uniform(1, 8)), float(g.uniform(1, 3)), tuple(g.uniform(0, L, 3)))
             for _ in range(natoms)]
    cell = np.diag([L, L, L])
    return make_system((ngrid,) * 3, cell, atoms, functional, 1e-10, device,
                       "cubic%d_L%g_s%d" % (ngrid, L, seed))


def dimer(seed=0, shape=(96, 96, 96), cell_lengths=(18.0, 18.0, 24.0), per_cluster=12,
          functional=1, device="cpu") -> System:
    """Dimer-like density: two clusters of 12 exponentials each (offsets
    N(0, 1.5 bohr) around centres separated by d in [3, 8] bohr along z),
    orthorhombic 18 x 18 x 24 bohr cell on a 96^3 grid."""
    g = _rng(seed)
    Lx, Ly, Lz = cell_lengths
    d = g.uniform(3.0, 8.0)
    atoms = []
    for cz in (0.5 * Lz - 0.5 * d, 0.5 * Lz + 0.5 * d):
        for _ in range(per_cluster):
            off = g.normal(0.0, 1.5, 3)
            c = (0.5 * Lx + off[0], 0.5 * Ly + off[1], cz + off[2])
            atoms.append((float(g.uniform(1, 6)), float(g.uniform(1.2, 3.0)), c))
    return make_system(shape, np.diag(cell_lengths), atoms, functional, 1e-10, device,
                       "dimer%dx%dx%d_s%d_df%d" % (shape + (seed, functional)))


def ligand_shell(seed=0, ngrid=192, L=36.0, functional=1, device="cpu") -> System:
    """Ligand-shell-like sparse density: a core of 40 exponentials within
    5 bohr of the centre (Z in [6, 8], zeta in [2, 3]) and 160 on 20 radial
    chains out to about 14 bohr (Z in [1, 6], zeta in [1, 2.5]); floor 1e-10,
    vacuum near 1e-8."""
    g = _rng(seed)
    c0 = np.array([L / 2] * 3)
    atoms = []
    for _ in range(40):
        v = g.normal(size=3)
        v *= g.uniform(0, 5.0) / np.linalg.norm(v)
        atoms.append((float(g.uniform(6, 8)), float(g.uniform(2, 3)), tuple(c0 + v)))
    for _ in range(20):
        u = g.normal(size=3)
        u /= np.linalg.norm(u)
        for s in range(8):
            rad = 6.0 + s * 1.1 + g.normal(0, 0.2)
            atoms.append((float(g.uniform(1, 6)), float(g.uniform(1, 2.5)), tuple(c0 + rad * u)))
    return make_system((ngrid,) * 3, np.diag([L, L, L]), atoms, functional, 1e-10, device,
                       "shell%d_s%d" % (ngrid, seed))


def uneven_batch(seed=0, count=64, sizes=(32, 48, 64, 80, 96, 128), functional_mix=True,
                 device="cpu", shape_seed=None) -> List[System]:
    """Independent systems with grids drawn per axis from ``sizes`` (non-cubic
    mixes), spacing h in [0.15, 0.30] bohr and 4-60 exponentials each.

    shape_seed: grids, spacings, exponential counts and functionals come from
    this seed and the exponentials themselves from ``seed`` (ranks of a
    weak-scaling run: the same work per rank, independent densities).  None,
    or equal to ``seed``: everything from ``seed``."""
    g = _rng(seed if shape_seed is None else shape_seed)
    ga = _rng(seed) if shape_seed is not None and shape_seed != seed else None
    out = []
    for i in range(count):
        shape = tuple(int(v) for v in g.choice(sizes, 3))
        h = g.uniform(0.15, 0.30)
        lengths = [s * h for s in shape]
        na = int(g.integers(4, 61))
        atoms = [(float(g.uniform(1, 8)), float(g.uniform(1, 3)),
                  tuple(g.uniform(0, 1, 3) * lengths)) for _ in range(na)]
        if ga is not None:      # g drew its atoms all the same, so its stream is seed-independent
            atoms = [(float(ga.uniform(1, 8)), float(ga.uniform(1, 3)),
                      tuple(ga.uniform(0, 1, 3) * lengths)) for _ in range(na)]
        fn = int(g.integers(1, 3)) if functional_mix else 1
        out.append(make_system(shape, np.diag(lengths), atoms, fn, 1e-10, device,
                               "batch%d_%dx%dx%d" % ((i,) + shape)))
    return out


def serving_requests(seed=0, count=2000, rate=200.0,
                     sizes=(48, 64, 80, 96, 112, 128, 160, 192, 224),
                     cap=(160, 192, 224)):
    """Poisson arrival times (mean ``rate`` per second) and request specs
    (grid shape sorted and capped at 160 x 192 x 224, 10-400 exponentials).
    Densities are built lazily by :func:`realise`."""
    g = _rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, count))
    reqs = []
    for i in range(count):
        shape = sorted(int(v) for v in g.choice(sizes, 3))
        shape = tuple(min(s, c) for s, c in zip(shape, cap))
        h = g.uniform(0.15, 0.30)
        na = int(g.integers(10, 401))
        reqs.append({"id": i, "arrival": float(t[i]), "shape": shape, "h": float(h),
                     "natoms": na, "seed": int(g.integers(0, 2 ** 31)),
                     "functional": int(g.integers(1, 3))})
    return reqs


def realise(req, device="cpu") -> System:
    g = _rng(req["seed"])
    lengths = [s * req["h"] for s in req["shape"]]
    atoms = [(float(g.uniform(1, 8)), float(g.uniform(1, 3)),
              tuple(g.uniform(0, 1, 3) * lengths)) for _ in range(req["natoms"])]
    return make_system(req["shape"], np.diag(lengths), atoms, req["functional"], 1e-10, device,
                       "req%d" % req["id"])


def hello_example():
    """The 1 x 2 x 2 example of the library section: rho = 1..4,
    sigma = 0.5..3.5, cell diag(1, 2, 2), vdW-DF1."""
    n = torch.tensor([1.0, 2.0, 3.0, 4.0], dtype=torch.float64).reshape(1, 2, 2)
    s = torch.tensor([0.5, 1.5, 2.5, 3.5], dtype=torch.float64).reshape(1, 2, 2)
    return System((1, 2, 2), np.diag([1.0, 2.0, 2.0]), 1, n, s, [], "hello")
