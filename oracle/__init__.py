"""FP64 CPU oracle for the recycled shifted-system solves.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute anything in this package: only ``tests/``, the smoke check and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow, readable NumPy implementation of what the paper
computes, written from the paper's text:

* ``operator``  -- the shifted operator (A + gamma E_k) of Eq. (blkeqn)/(shift),
  matrix-free, and the edge-preserving weights.
* ``minres``    -- recycled MINRES of Section 2.3 / Eq. (minShift), with plain
  MINRES (Paige-Saunders) as the special case K = [].
* ``recycle``   -- the principal recycle space (Sections 4.1, 5.1, 5.2,
  Algorithm "Stabilized U"), the local spaces (Algorithms "interior",
  "updatelocal", "updatelocalV2") and the per-shift solves of one outer step
  (Algorithm "Shifted Recycling Algorithm").
* ``outer``     -- the L-curve corner and the reweighting outer loop.
* ``adjoint``   -- adjoint solves and the gradients of a loss of the solutions
  with respect to the shifts and the weights.

It shares no code with the CUDA path. Its only shared dependency is the seeded
input generator ``synth`` (which holds no arithmetic of the method).

Pinning: every function here is pinned by a ``-m "not gpu"`` test against
something other than itself (dense matrices built from the definitions, dense
solves, the generalized-eigen closed form, SciPy's MINRES, brute-force
least squares over explicit bases, constructed inputs with known answers).
Parity unpinned: the per-shift matvec counts against the paper (its counts
exist only as figures that are not reproduced in the text).
"""
