"""FP64 CPU oracle for the ADI isogeometric Maxwell time stepper.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The GPU library (``paper_2103_06998_gb300``) never
imports it, and this package never imports the GPU library: the two share no
code.  Inputs reach both sides from ``paper_2103_06998_gb300.inputs`` (seeded
generators only, none of the method's arithmetic), passed in by the caller.

The oracle is a plain, slow, obviously-correct restatement of the method of
Paszynski, Los and Munoz-Matute, "Alternating directions implicit higher-order
finite element method for simulations of time-dependent electromagnetic wave
propagation in non-regular biological tissues" (arXiv 2103.06998):

* ``bspline``      open uniform knots, Cox-de Boor basis, 1D matrices M, S, A, B
                   ("Variational formulation", definitions after eq. discrete4).
* ``banded``       1D operators along one axis of a 3D coefficient array and
                   Gaussian elimination (no pivoting) of banded line systems.
* ``material``     per-test-function material ("Incorporating non-regular
                   material data", the hat values), conductivity coefficients,
                   explicit CFL limit.
* ``maxwell_adi``  the four sub-solves of one time step (eqs. scheme1a-1d,
                   weak1-weak4, discrete1-discrete4, dupa1ab, Appendix order).
* ``manufactured`` the manufactured solution u_A and L2 / H(curl) norms
                   ("Numerical code verification with manufactured solution").
* ``convnet``      the learned coarse-step corrector (not in the paper): 3D
                   convolution net, MSE, gradients, Adam, input features.

Parity status per function is listed in each module header.  Every function is
pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py`` except where a
header says "parity unpinned".
"""
