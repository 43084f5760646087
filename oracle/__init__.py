"""FP64 CPU oracle for the truncated-solver disconnected-loop path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.  It shares no code,
table or constant generator with the CUDA library; the only inputs both sides
receive are the seeded gauge links (and test spinors) made by
``paper_1401_6750_gb300.synth``, which holds none of the method's arithmetic.

Everything here is plain numpy in complex128, written from the definitions the
paper relies on (arXiv:1401.6750):

* ``gamma``    -- Euclidean Dirac matrices (chiral basis) and the 16 insertion
                  matrices Gamma_g (Sec. 2.1.1 "ultra-local ... insertions").
* ``lattice``  -- site order, neighbour shifts and the temporal boundary sign.
* ``dirac``    -- twisted-mass Wilson operator M, M^dagger, M^dagger M (Eq. 1).
* ``solver``   -- conjugate gradient on M^dagger M for Eq. 1 (Sec. 2).
* ``dense``    -- dense matrices, LU inverse and exact traces (small lattices).
* ``philox``   -- Philox4x64-10 (Salmon et al., SC'11) and Z4 volume sources
                  (Sec. 2: "random stochastic sources").
* ``momenta``  -- the p^2 <= 9 momentum list (Sec. 2.1.1, Sec. 2.3).
* ``contract`` -- one-end-trick loop densities for the 160 insertions and the
                  momentum projection per timeslice (Sec. 2.1.1, Sec. 2.2).
* ``tsm``      -- the truncated-solver combination (Sec. 2.1).
* ``freefield``-- unit-gauge closed forms in momentum space (pins only).

Parity status: every function is pinned by a ``-m "not gpu"`` test against
something other than itself (closed forms, numpy library routines, algebraic
identities, brute force).  Parity unpinned: the absolute normalisation of the
paper's own published loop values -- the paper prints none.
"""
