"""CPU oracle for the FIND selected-inversion path (float64 / complex128).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path and never imports it; the product path never imports this.

Modules:
  problem -- H, lead self-energies (sine-mode closed form), A, Sigma<
  dense   -- O-dense: G = A^{-1}, G< = G Sigma< G^H, bond currents
  find    -- O-find: the paper's upward / downward / leaf procedures

Parity status: every function is pinned by ``tests/test_oracle_*.py``
(dense inverse on small meshes, closed forms of the clean wire, the eta
identity, current continuity, Landauer transmission, tree independence,
symmetry invariants, and a non-symmetric general-A check).  No function is
left "parity unpinned".
"""
from . import problem, dense, find  # noqa: F401
