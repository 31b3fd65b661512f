"""CPU oracle for the O(a)-improved Wilson-Dirac block solvers (TEST INFRASTRUCTURE).

This package is a plain, slow, FP64 numpy restatement of what the method
computes.  It is written from Sakurai, Tadano and Kuramashi,
"Application of block Krylov subspace algorithms to the Wilson-Dirac equation
with multiple right-hand sides in lattice QCD" (arXiv:0903.4936):

* ``gamma``   - the Euclidean gamma matrices as printed, sigma_mu_nu (Section 2)
* ``clover``  - the clover-leaf field strength F_mu_nu (Section 2)
* ``dirac``   - D_W applied to a block of L spinor columns, Eq. (wd-op)
* ``dense``   - the dense N x N matrix of D_W on small lattices
* ``solvers`` - scalar BiCGSTAB, block BiCGSTAB and block BiCGGR (Section 3)
* ``evenodd`` - the even-odd (Schur complement) form of the same system, a
  reordering that is not in the paper, defined from the pieces above

It is test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference arm may import it.  The product
path (``paper_0903_4936_gb300``) never imports it, and it shares no code with
the CUDA kernels; the only common module is ``synth`` (seeded inputs).
"""
from . import gamma, clover, dirac, dense, solvers, evenodd  # noqa: F401
