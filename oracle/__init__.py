"""Plain FP64 CPU oracle of the MOL^T Cahn-Hilliard hot path (arXiv 1611.04214).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
product path (the CUDA library and its binding) never imports it, and this
package never imports the product path: the two share no code.

The oracle is slow and literal on purpose.  Each function restates one passage
of the paper (cited in its docstring) in FP64 numpy, in the paper's order and
notation, with no blocking, fusion or reordering:

* ``weights``   - local quadrature weights of the fast convolution (Sec. 3.2)
* ``helmholtz`` - the 1D modified-Helmholtz inverse L^{-1} = (I - c d_xx)^{-1}
                  by particular + homogeneous solution (Eq. L_Inverse, Iu, IL,
                  IR, homogeneous)
* ``solver``    - stage parameters, the 1D and 2D fixed-point stage solves
                  (Eq. CH_BE_fixed2_factor, CH_BE_fixed_complete, Sec. 5.1),
                  time schemes (BE, BDF2, BDF3, SDIRK2, SDIRK3, SDC2) and the discrete
                  energy / mass.
* ``adaptive``  - adaptive step-size control (Algorithm 1) with the Richardson,
                  BE-SDC2 and BE-BDF2 LTE estimates.
* ``vch``       - the vector (three-phase) model of Eq. CH_vector: potential,
                  stage parameters of Eq. CH_vector_fixed1/2, stage solve, BE and
                  BDF2 steps and energy (Sec. 5.2).
* ``split3d``   - the splitting of Sec. 5.1 carried to three dimensions (the
                  extension the paper remarks on), BE and BDF2.
* ``fch``       - the sixth-order model of Eq. FCH0 / FCH in 1D and 2D, BE by
                  completing the cube (Eq. FCH_BE, with the PDE's signs); in 2D with
                  the splitting of Sec. 5.1 for the three equal factors.

Readings of passages the paper leaves open are listed in each docstring.
"""
