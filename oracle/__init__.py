"""Plain, slow FP64 CPU oracle for the even-odd preconditioned Moebius domain-wall
fermion (MDWF) propagator solve of arXiv:1810.01609.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA
library (no kernels, headers, helpers, tables or constant generators).

The paper (Sec. "Current State of the Art") names the operator -- the Moebius
domain-wall Dirac operator on L^3 x T x L5 x Nc x Ns, a radius-one stencil with small
dense diagonal blocks -- the solver -- conjugate gradient on the normal equations with
red-black (even-odd) preconditioning -- and the Feynman-Hellmann propagator, but prints
no formula, basis or convention.  The readings taken here are listed in each module
and pinned by closed forms, brute force and symmetries in ``tests/test_oracle_*.py``.

Modules
  gamma    chiral gamma basis, projectors, charge conjugation
  dirac    Wilson hop, D_W, s-direction operators, 5D Moebius operator, even-odd pieces
  solve    CGNR on M_pc (and on the full 5D operator), even-odd solve
  hadron   4D source injection / projection, Feynman-Hellmann source, nucleon 2-pt
  storage  FP16 (+ per-site norm) / BF16 / FP32 storage quantisers
  sample   site-sampled evaluation of the same operators for lattices too large
           for a full oracle pass
"""
from . import gamma, dirac, solve, hadron, storage, sample  # noqa: F401
from .dirac import MobiusParams  # noqa: F401
