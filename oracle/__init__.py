"""Plain FP64 CPU oracle of the relativistic lattice Boltzmann (RLBM) step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, links or calls anything here, and this package imports nothing from
the product.

The oracle follows Gabbana, Simeoni, Succi, Tripiccione, "Relativistic Lattice
Boltzmann Methods: Theory and Applications" (arXiv:1909.04502):

* ``lattice``  -- stencils, quadratures (App. H), orthonormal polynomials
  (App. F, and Gram-Schmidt of Sec. 5.2 for order 3), projections (App. G and
  the Z-tensor integrals of App. B), the quadrature search of Sec. 5.3.
* ``physics``  -- equation of state (Eq. eos-ddim, Eq. defG), Landau-frame
  eigen-solve (Sec. 4), Chapman-Enskog shear viscosity (App. C).
* ``scheme``   -- the per-cell algorithm of Sec. 6.2 (moments, Landau solve,
  n, T, equilibrium, relaxation) and streaming (Eq. discrete-rbe), plus the
  off-lattice bilinear streaming and free-flow ends described in this
  package's readings.

Everything is plain numpy in float64, vectorised over lattice cells only;
library primitives used as steps are LAPACK ``eig``/``lstsq`` and scipy's
Bessel functions.  Readings of places where the paper is silent or garbled
are stated in the docstring of the function that takes them.
"""
