"""FP64 CPU oracle for the disaggregated D3Q19 lattice-Boltzmann hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, links or runs anything in this package; only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` do.

The oracle is deliberately the plain method: full virtual-box numpy arrays,
one vectorised pass per lattice direction, no blocks, no grouping, no fusion
and no reordering.  The paper (Sec. 2, Definition; Sec. 4; Sec. 5) states
that disaggregation only changes how voxels are mapped to memory and which
kernel processes them, so every disaggregated layout must reproduce this
plain computation.  The paper names the lattice-Boltzmann ingredients (D3Q19,
BGK, bounce-back, regularized boundaries, explosion/coalescence: Sec. 6,
Sec. 6.2, Sec. 6.3) without writing their formulas; each module states the
reading it implements.

Modules
  lattice   D3Q19 velocity set, weights, opposite table, equilibrium.
  lbm       one time step on a virtual box (streaming, bounce-back,
            regularized velocity / pressure boundaries, BGK / regularized
            collision), moments, conservation sums, Taylor-Green and
            Poiseuille closed forms.
  layout    brute-force construction of the sparse block tables (active
            blocks, boundary-first Morton numbering, neighbour table).

Pins (``tests/test_oracle_pins.py``) tie every function here to the lattice
invariants, exact conservation laws, closed-form flows and fixed points.
"""
