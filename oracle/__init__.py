"""CPU FP64 oracle for the low-rank Poisson solve of arXiv:1306.2150.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The CUDA library never calls it and shares no code
with it: no kernels, headers, tables, constant generators or pre/post-processing.

Everything is plain numpy (float64) written from the paper:

* ``poisson_lowrank`` -- the operators of Section 2, the sine-transform
  diagonalisation of Section 4.1 (Eq. flr:diag), the frequency-space symbol of
  Section 4.2 (Eq. flr:div), the full-grid solve, a dense LU solve, the cross
  approximation in frequency space (Section 4.2), the rounding of Section 3 and
  the low-rank solve built from them, plus exact error evaluation by Parseval.
* ``maxvol`` -- the maxvol row selection the cross of Section 4.2 cites.
"""
from . import poisson_lowrank  # noqa: F401
