"""FP64 CPU oracle for COLA with scale-dependent growth (Winther et al., arXiv:1703.00879).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of the method in NumPy/SciPy double precision.  It is
imported only by the tests, by ``__graft_entry__.smoke()`` and by the CPU
baseline leg of ``bench.py``.  The CUDA library never calls it and shares no
code with it; the only common input is the configuration record in
``workloads.py`` (the white noise is drawn by each side from its own Philox
implementation).

Modules, each following the paper passage named in its docstring:

* ``background`` - LCDM expansion, super-comoving time tau, kappa (Sec. 1, Sec. 3)
* ``models``     - mu(k,a), gamma_2, screening factors (Sec. 5, Sec. 6, App. B, App. C)
* ``growth``     - scale-dependent 1LPT/2LPT growth ODEs and tables (Sec. 4)
* ``power``      - Eisenstein-Hu no-wiggle linear power spectrum, sigma_8
* ``philox``     - Philox-4x32-10 counter generator and Box-Muller normals
* ``ics``        - Gaussian field and 2LPT potentials (Sec. 3.2, Eq. lcdm2lpt)
* ``pm``         - CIC mass assignment, Poisson/screened field solve, force, P(k)
* ``cola``       - COLA kick-drift-kick stepper in the LPT frame (Sec. 2, App. A)

Parity status of each function is stated in its module header; "parity
unpinned" marks the functions no closed form or printed value pins.
"""
