"""FP64 CPU oracle for the Galerkin boundary-integral method of active spheres.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything here.  The CUDA path in ``paper_1411_0278_gb300`` shares no code,
table or generator with this package and never imports it.

Modules: ``tensors`` (STF projectors, tensorial harmonics, packed basis, mode
embeddings), ``taylor`` (exact truncated Taylor series of |rho|^nu),
``galerkin`` (pair and self elements, dense system, LU solve, superposition),
``quadrature`` (brute-force surface integrals used only to pin the above),
``dynamics`` (forward-Euler trap update), ``flow`` (the flow field of the Galerkin
representation at points in the fluid, by surface quadrature), ``mlp`` (features,
network, loss, gradient and Adam step of the learned near-field correction).

Parity status: every function is pinned by tests/test_oracle_pins.py and
tests/test_oracle_mlp_pins.py against
closed forms, textbook limits or brute-force quadrature; none is "parity unpinned".
"""
