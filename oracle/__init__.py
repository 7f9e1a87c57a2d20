"""CPU oracle for the mixed-precision sketch-and-precondition least-squares method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, links or runs anything here, and this package imports nothing from
the product path.

Every function is a plain, slow, obviously-correct restatement of the method
of Carson & Dauzickaite, "Mixed precision sketching for least-squares problems
and its application in GMRES-based iterative refinement" (arXiv 2410.06319):

* ``rng``      -- Philox4x32-10 counter stream and the FP64 Box-Muller
                  Gaussian used for the sketch matrix (Sec. 2: Gaussian
                  embedding with N(0, 1/s) entries; Sec. 5: Omega = s^-1/2 G).
* ``sketch``   -- Algorithm 1 (the sketch) (Y = Omega A in u_s), with the one-sided
                  power-of-two column scaling of Sec. 3.2.
* ``sparse``   -- the sparse sign embedding of Sec. 2 as the sketch: zeta
                  signed rows per data row (Philox, Floyd's sampling), exact
                  fixed-point sums.
* ``qr``       -- Algorithm 1 (the QR of the sketch) (Householder QR of Y; R only) and the
                  sketch-and-solve start x_s = R^-1 Q^T Omega b (Sec. 4).
* ``lsqr``     -- Algorithm 2 (the LSQR start): LSQR right-preconditioned by R.
* ``fgmres``   -- Algorithm 2 (the FGMRES solve): split-preconditioned FGMRES, Eq. (1.2).
* ``lsir``     -- Algorithm 2 (augmented-system iterative refinement) with
                  the precision-escalation rule of Sec. 5.
* ``dd``       -- products beyond double (exact splits and sums, rounded to
                  double-double) for the escalated FGMRES of Sec. 5 with u
                  double (u_A = u_L = u_R = quad).
* ``exact``    -- double-double residuals (Dot2) and a refined reference
                  solution x*, r* (the role of the 64-digit solve of Sec. 5).
* ``theory``   -- closed forms used as pins (Sec. 2 identities, Eq. 4.1,
                  Marchenko-Pastur limits of kappa(A R^-1)).
* ``workload_counts`` -- the oracle's iteration counts on the m = 1e5,
                  n = 500 workload, which the reference leg of bench.py
                  scales its sampled per-iteration times to.

Arithmetic is FP64 unless a function takes an explicit working dtype (the
paper's precisions u, u_A, u_L, u_R are parameters of the method).

Parity unpinned: nothing.  Every function has at least one pin in
``tests/test_oracle_*.py`` against values the mathematics or the paper fixes.
"""
