"""Plain, slow, FP64 CPU oracle for the Lippmann-Schwinger method of
Eikrem, Naevdal and Jakobsen, "Iterative solution of the Lippmann-Schwinger
equation in strongly scattering acoustic media by randomized construction of
preconditioners" (arXiv:2005.01372).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline / reference legs of ``bench.py`` may import it.  The
library (``paper_2005_01372_gb300``) never imports it and shares no code with
it: the two meet only through the seeded velocity models of
``paper_2005_01372_gb300.media`` and through the published conventions listed
below, each implemented separately on each side.

Modules (each function cites the passage it follows):

* ``green``    -- contrast (Eq. 1), cell-integrated Green's function, its
                  block-Toeplitz table, even extension and spectrum (Sec. 2.2).
* ``operator`` -- G0 V u by dense O(n^2) summation and by zero-padded FFT
                  convolution (Eq. 4, Sec. 2.2), the adjoint, the residual.
* ``solve``    -- direct LU solve (Eq. 5-6), Born series (Sec. 2.2),
                  preconditioned scattering series (Eq. 10-11, Eq. 13-14),
                  flexible GMRES.
* ``philox``   -- Philox4x32-10 counter-based generator (Salmon et al.,
                  SC'11) and Box-Muller complex Gaussians for the probes.
* ``sketch``   -- randomized range finder (Algorithm 1, Algorithm 2) and its
                  SVD truncation.
* ``smw``      -- the simple low-rank preconditioner (Eq. 12).
* ``hodlr``    -- HODLR tree, randomized construction (Sec. 2.4, Fig. 1),
                  recursive block inversion with randomized recompression,
                  matrix-vector product.

Conventions fixed here (readings of the paper where it is silent):

* unknowns ordered in vertical strips, linear index ``ix * nz + iz`` (Sec. 2.4);
* time convention exp(-i w t), G0(r) = (i/4) H0^(1)(k0 r);
* each cell is integrated as the disk of equal area (radius h / sqrt(pi)), so
  the cell volume of Eq. 4 lives inside the Green table and V = diag(chi);
* the even circulant extension of the Green table to 2nz x 2nx, with index N
  holding the offset-N value, stands in for the extension of Nowak et al.
  (2003) that the paper cites but does not spell out;
* "T" in the paper is the conjugate transpose (Sec. 2.3).
"""
