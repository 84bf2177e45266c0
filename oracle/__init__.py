"""FP64 CPU oracle for primed PCA (pPCA) -- TEST INFRASTRUCTURE ONLY.

Only the test suite (``tests/``), ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may import this package.  The product
library (``paper_2109_03709_gb300``) never imports, links or calls it, and the
two share no code: this package is a plain, slow, obviously-correct restatement
of the method in double precision, written from the paper.

Contents (each function cites the passage it follows):

* O1 ground truth -- the principal directions are the eigenvectors of X^T X
  (Section 1); diagonalised with this package's own cyclic Jacobi
  (``jacobi.c``).
* O2 the pPCA step given a primed basis V (Algorithm 1, steps 2-5;
  Section 4.2 on the variance restricted to S).
* O3 the three primers: block power / simultaneous iteration (Section 2.1),
  Oja's generalised (Sanger) rule (Section 2.2), EigenGame utilities
  (Section 2.3, Eqs. 1-3) with SGD + Nesterov momentum 0.9 (Section 5).
* O4 metrics: angle, longest correct eigenvector streak (Section 5.3),
  principal angles, variance captured (Section 5.3 footnote).
* The e4m3 / bf16 codecs used to read stored low-precision data exactly.

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, brute force, the paper's worked examples and invariants.  Functions with
no such pin say so in their docstring ("parity unpinned").
"""
from .core import *  # noqa: F401,F403
from .core import __all__  # noqa: F401
