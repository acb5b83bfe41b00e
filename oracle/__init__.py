"""Plain FP64 CPU oracle for the RBM variational Monte Carlo hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import, call, link or run
anything under ``oracle/``.  The product package never does, and the two share
no code: the only thing both sides consume is the seeded input generators in
``paper_2112_10526_gb300.inputs``, which hold none of the method's arithmetic.

Layout:
  nk_oracle.c  per-configuration definitions in C (ln psi, local energy,
               log-derivatives, Philox4x64-10, chain initialisation,
               Metropolis chains with forced-follow replay);
  core.py      ctypes binding of the C part plus the sample statistics, force,
               QGT, SR linear solves and update in numpy (Sec. 3.3, 3.5, 4.1,
               App. B of the paper);
  exact.py     exact enumeration over all basis states and exact
               diagonalisation from Kronecker products of Pauli matrices;
  symm.py      the symmetric RBM (RBMSymm, Sec. 5): ln psi and
               log-derivatives over a site-permutation group, SR step
               through the equal plain RBM with tied parameters;
  holo.py      the complex holomorphic RBM, its Metropolis chains on the
               real oracle's Philox streams, its force and QGT (exact or
               sampled) and the TDVP equation of motion with Euler and Heun
               steps (Sec. 4.3), in complex128.

Parity pins are in tests/test_oracle_*.py.  A function without an external
pin would say "parity unpinned" in its docstring; none does.
"""
from .core import *  # noqa: F401,F403
