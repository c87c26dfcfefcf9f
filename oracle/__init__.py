"""FP64 CPU oracle for W-projection gridding and degridding.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call,
link or execute anything in this directory; only the tests, the smoke check
and the CPU-baseline leg of the benchmark use it.  It shares no code with
the CUDA path: it has its own prolate-spheroidal solver, its own quadrature,
its own kernel tables, its own index selection and its own (C) gridding
loops.

Citations name the thesis' sections and equation / algorithm labels
(the thesis numbers them only through LaTeX labels):

* Section 1.2, Eq. (measurmentequation): the measurement equation, the
  forward model that degridding approximates.
* Section 1.3, Eqs. (gw), (v00): the w-screen g_w, its inverse and the
  plane-to-plane convolution that W-projection (Section 1.7.1) folds into
  the gridding convolution function (GCF).
* Section 1.7, Eq. (ID): the dirty image that gridding + IFFT + correction
  approximates.
* Section 2.3, Algorithm (convgridding), and Section 2.4.5, Algorithm
  (convgriddingoversampling): gridding with a beta-oversampled GCF table.
* Section 2.3.1: the Bounded Records Assumption (records whose footprint
  leaves the grid are ignored).
* Section 2.3.6 / 2.4.5, Eqs. (cco), (hco): what oversampling does to the
  GCF and the corrector.
* Section 2.4.2, Algorithm (equivalentalgo): NN interpolation onto the
  beta-fine grid followed by convolution and decimation equals gridding
  with the oversampled table (an exact identity used as a pin).

Modules:

* ``index``   -- uvw (metres) -> pixel k, oversampled offset o, w-plane p,
                 conjugation flag and the bounded-record flag.
* ``pswf``    -- the zeroth-order prolate spheroidal wave function, the
                 taper (Section 2.3.4).
* ``wkernel`` -- w-projection kernel tables (Fourier transform of
                 taper x w-screen, sampled on the beta-oversampled grid) and
                 the grid corrector.
* ``cgrid``   -- plain FP64 gridding / degridding loops in C.
* ``image``   -- centred inverse DFT of a grid, the correction step, and the
                 brute-force non-uniform DFTs of Eq. (ID) and
                 Eq. (measurmentequation).

Where the thesis is silent the oracle takes the readings listed in the
repository's design notes; each module header repeats the ones it uses.
"""
