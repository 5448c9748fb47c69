"""CPU FP64 oracle for the LSMS Kubo-Greenwood conductivity hot path (arXiv 2311.12134).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may import
this package.  It shares no code with the CUDA library in
``paper_2311_12134_gb300`` and imports nothing from it: inputs arrive as plain
NumPy arrays made by the seeded generators, and every function here is a plain,
slow restatement of the paper's equations in float64 / complex128.

Modules and the passages they follow
-----------------------------------
``sph``        real spherical harmonics Y_L (explicit associated-Legendre
               polynomials) and real Gaunt coefficients (quadrature); the
               angular basis of Sec. II.A (G expressed over L = (l, m)).
``hankel``     spherical Hankel functions h_l^(1), h_l^(2) by their finite
               closed form.
``structure``  the free-electron propagator g^{nm}_{LL'}(z) of Eq. (tau-inverse).
``liz``        the local interaction zone of Sec. II.A (Fig. 1) by brute force.
``kkr``        M = T^{-1} - g and the scattering-path blocks tau^{n0}, tau^{0n}
               of Eq. (tau-inverse), by dense LAPACK solves.
``kubo``       the LSMS Kubo-Greenwood traces (Eq. lsms-conductivity-formula),
               the four-combination consolidation (Eq. sigma-tilde-consolidation),
               the resistivity tensor, and the dipole current-matrix model.
``grad``       d sigma / d t^{-1}_i through explicit full inverses
               (d tau = -tau dM tau), with no adjoint trick.

Parity status: every function above is pinned by tests in
``tests/test_oracle_pins.py`` (closed forms, special cases, invariants,
brute-force comparisons).  What stays parity-unpinned is the absolute scale of
sigma against experiment: the current matrices are a synthetic model and the
paper's potentials are not available.
"""
