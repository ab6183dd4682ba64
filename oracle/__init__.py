"""FP64 CPU oracle of the FFT-preconditioned finite-element homogenisation solver.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the CUDA path is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import or run it; the product path (the C-ABI library and its Python binding) never does, and the
two share no code.  Inputs come from the seeded generators in
``paper_2203_02962_gb300.inputs`` (random draws and geometry only, none of the method's
arithmetic), which both sides receive as plain arrays.

Modules:
  fem      -- D, W, C, K = D^T W C D, b = -D^T W C e, <sigma> (Sec. 3, Eq. lin_system, App. A)
  solvers  -- Algorithm 2 symbol + pseudo-inverse (Sec. 5.2-5.3), preconditioner apply
              (Eq. M_inverse), dense/sparse/CG solves and the paper's PCG (Sec. 4.1, Sec. 6)
  newton   -- Algorithm 1 (Newton with per-step reference reassembly) for a power-law conductivity
  unet     -- the periodic 3-D U-Net of the learned warm start (an addition to the paper's method):
              forward pass, chain-rule gradient and Adam, channel-first FP64

Every function is pinned by ``tests/test_oracle_pins.py`` against facts the paper and the
mathematics fix (closed forms, invariants, exact laminate results, brute force on tiny grids).
"""
from . import fem, newton, solvers, unet  # noqa: F401
from .fem import Grid  # noqa: F401
