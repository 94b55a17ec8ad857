"""FP64 CPU oracle for the transcorrelated (TC / BITC) two- and three-body operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA path (``paper_2302_07420_gb300/csrc``) and never reads anything the CUDA
path produced.

What it computes (M. Ochi, "TC++: First-principles calculation code for solids
using the transcorrelated method", arXiv:2302.07420):

* ``cell``      -- cell, Gamma-centred k mesh, plane-wave spheres, FFT box,
                   Gygi-Baldereschi constant (Sec. 2.5, Eqs. correction2, aux).
* ``kernels``   -- Fourier transforms of u, lap u, (grad u)^2 and V_2a
                   (Sec. 2.6.3 and Appendix B).
* ``operator``  -- the two-body terms 2ah, 2bh1, 2bh2, 2ax, 2bx1, 2bx2 and the
                   three-body terms 3a1-3a4, 3b1-3b6 (Algorithms 1-12), with the
                   divergence corrections for k on the SCF mesh
                   (Eqs. divcorr_2ax_scf, divcor_3a2_first/second and their
                   density-matrix forms, 3b6_div_scf1/2/3), the left operator and
                   the TC pseudo-energy (Eqs. EtotTC / EtotBiTC).
* ``direct``    -- a second backend for ``operator`` that replaces every FFT by
                   direct cyclic sums in reciprocal space (brute force, tiny grids).
* ``band``      -- the operator at band-structure k-points off the SCF mesh
                   (partners on the mesh) with the band forms of every
                   divergence correction (Eq. divcorr_2ax_band, the grad-u
                   forms of Eq. correction_nabla, Eqs. 3b6_div_band1/2/3).
* ``ewald``     -- Ewald lattice sums (the Madelung potential and its phased
                   form), used only to pin the divergence-correction constants.

Every floating-point quantity is FP64.  Parity status of each function is stated
in its module header.
"""
