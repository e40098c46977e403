"""Plain, slow, FP64 CPU oracle for the SR-CPM electrode-charge path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The CUDA
library never calls it, and it never imports the CUDA package: the two share no code.

Every function follows a passage of Li, Wang, Liu & Jiang, "A Simple and Efficient
Lattice Summation Method for Metallic Electrodes in Constant Potential Molecular
Dynamics Simulation" (arXiv 2111.06704), cited by section and equation:

* ``ewald``   -- k-vector table, the Gaussian Ewald interaction matrix E (Eq. 22-23 with
  the slab correction Eq. 39), the electrolyte potential b^sol (Eq. 25), and the
  neutral-equivalent form used by the GPU path (Eq. 29-30, 39).
* ``solve``   -- the bordered electroneutral system (Eq. 29 + 34), the two-step method
  (Eq. 35, S8-S9), the S matrix (Eq. 33), and plain / preconditioned CG (Sec. III B 2).
* ``precond`` -- the PCG-DC preconditioner (Eq. 36) and p_gap (Eq. 37).
* ``mlp``     -- the per-atom initial-guess network (project-defined; the paper is
  silent on it) in FP64 with hand-written backpropagation.
* ``gcd``     -- fixed total charge per electrode (galvanostatic charge-discharge,
  Eq. S14-S24): capacitance coefficients and the two-step GCD charges; pinned by
  ``tests/test_oracle_gcd.py``.
* ``forces``  -- forces on the ions from the electrode's Gaussian charges (Eq. S25 inside
  the Ewald form of Eq. 22 / 25); pinned by ``tests/test_oracle_forces.py``.
* ``precond.sparsified_inverse`` -- the PCG-Normal / PCG-Full preconditioners (Fig. 6a);
  pinned by ``tests/test_oracle_pcg_variants.py``.

Parity status: every function is pinned by ``tests/test_oracle_pins.py`` (Madelung
constants, the 2D lattice constants and Gaussian widths of Table 1, brute-force
real-space lattice sums of Eq. 17 for E and for b^sol, the closed-form charges of a
two-sheet capacitor, splitting-parameter independence, three routes to the neutral
charges, the Fig. 2 neighbour count) except where a function's docstring says "parity
unpinned".
"""
