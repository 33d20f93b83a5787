"""FP64 CPU oracle for the adiabatic-master-equation (AME) trajectory path.

TEST INFRASTRUCTURE ONLY. Nothing in the product library imports, links or
calls this package; only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it. It shares no code with the CUDA path:
its eigensolver is LAPACK through numpy, its Lamb-shift quadrature is
QUADPACK through scipy, its propagators are scipy matrix exponentials, and
its random streams come from its own Philox implementation.

Modules (each function cites the passage of arXiv:1710.03431 it follows):
  philox        Philox4x64-10 counter generator and the per-trajectory stream layout
  model         TFIM Hamiltonian (Sec. V, Eq. H_S), schedule, eigensystems,
                degenerate manifolds and Bohr-frequency classes (Sec. II, Eq. Lindblad2)
  bath          Ohmic rates gamma(omega) (Sec. V) and the Lamb shift S(omega)
  ame           density-matrix AME (Sec. II, Eqs. ME2-H, ME2-L), split-exact
  trajectories  serial waiting-time sampler (Sec. IV; App. B.1, Eq. Pi(t); App. C)

Readings of the paper that both this oracle and the CUDA path follow are
listed in the functions that implement them.
"""
