"""Plain FP64 CPU oracle for the particle-mesh step with massive-neutrino particles.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run it.  It shares no
code, tables or constants generator with the CUDA path.

Every function restates, in FP64 numpy/scipy, one step of the method of
Bayer, Banerjee & Feng, "A fast particle-mesh simulation of non-linear
cosmological structure formation with massive neutrinos" (arXiv 2007.13394),
or of the particle-mesh machinery the paper inherits from FastPM.  Library
primitives used as single steps: numpy's FFT (rfftn/irfftn), numpy's stable
argsort, numpy's bincount (fixed-order sums), scipy quadrature, scipy's ODE
integrator and root finder.  Nothing is blocked, fused or reordered beyond the
definition it follows.

Modules
-------
background  E(a) with photons, massive neutrinos (the F(y) integral), CDM and
            Lambda; the linear growth ODE; FastPM kick/drift coefficients.
neutrinos   Fermi-Dirac shell tables (equal area under g(q) = q f(q)), the
            effective distribution for non-degenerate masses, Fibonacci
            directions, neutrino site lattice.
pm          fixed-point positions, the (tile, face-class) sort key, CIC paint,
            Green's function, spectral gradient, CIC readout, kick, drift,
            one KDK step, the binned power spectrum.
ic          BBKS spectrum, sigma_8 normalisation, Zel'dovich initial
            conditions for CDM and neutrino sites.
ewald       brute-force periodic Ewald sum of the force of one point mass.

Parity status: every function is pinned by a test in ``tests/test_oracle_*.py``
against a closed form, a limit, an invariant or brute force.  The Fibonacci
directions are pinned by the properties their golden-angle lattice fixes
(equal-area zones, packing distance, Fibonacci parastichies), which reject
spirals with another turning angle.
"""
