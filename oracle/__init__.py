"""FP64 CPU oracle for the vdW-DF nonlocal correlation (RPS FFT method).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import, call, link or run
anything in this package.  The product path (the CUDA library and its Python
binding) never imports it, and this package never imports the product.

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except where its docstring says "parity unpinned".

``oracle.spin`` holds the spin-polarised form (q0 of both spins, energy and
four potentials).
"""
from . import spin
from .vdw import (Params, Oracle, calculate, q_mesh, spline_basis_d2, spline_basis,
                  q0_of, pw92_eps_c, saturate, phi_dion, kernel_table, kernel_at,
                  radial_transform, kabs_grid, cell_volume, pair_list, DF1, DF2,
                  oracle_threads)

__all__ = ["Params", "Oracle", "calculate", "q_mesh", "spline_basis_d2", "spline_basis",
           "q0_of", "pw92_eps_c", "saturate", "phi_dion", "kernel_table", "kernel_at",
           "radial_transform", "kabs_grid", "cell_volume", "pair_list", "DF1", "DF2",
           "oracle_threads"]
