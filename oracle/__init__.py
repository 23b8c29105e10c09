"""FP64 CPU oracle for the implicit constraint-resolution hot path.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the
smoke check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py``
may import or run anything in this package.  It shares no code with the GPU
library (no kernels, headers, helpers or constants) and neither imports the
other; both consume inputs from the seeded generator ``scenegen``.

What it computes, each function citing the passage it restates:
  * ``delassus``: the mapping matrix H (Eq. "geometrical mapping", barycentric
    G), the direction matrix C (Eq. "jacobian directions"), J = C H
    (Eq. "isolate directions"), the Delassus operator W = J A^-1 J^T formed
    directly (Eq. "schur complement", Alg. 2 step 2), the mapping compliance
    W_H = H A^-1 H^T and the reformulated W = C W_H C^T
    (Eq. "schur complemnt reformulated").
  * ``pgs``: projected Gauss-Seidel (Eq. "PGS", Alg. 1) with a
    Signorini / Coulomb local solve (Eqs. "signorini's law", "coulomb's law")
    and the complementarity and friction-cone residuals.
  * ``newton``: the standard recursive scheme (Alg. 2) and the fast scheme
    (Alg. 3) with the proximity update of Eq. "recursive motion correction 7"
    and the summed correction of Eq. "recursive motion correction 3".
  * ``reach``: the supernodes each column of H^T reaches in the elimination
    tree (the nonzero structure of L^-1 H^T).

Every function works in FP64.  The PGS is written as plain Python loops over
contacts with NumPy row products, in the paper's order.
"""
