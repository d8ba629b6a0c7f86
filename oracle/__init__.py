"""FP64 CPU oracle for the TaCauchy hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct numpy/scipy implementation of what the GPU
library computes, written from the paper (TaCauchy, Sec. III-B/III-C,
Eq. 1-8, Algorithms 1-2) and from the incremental-potential-contact method it
configures (Li et al. 2020, "Incremental Potential Contact").  It shares no
code with the CUDA path and imports nothing from it.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path never calls it.

Modules
  material  Eq. 1 Lame parameters; stable Neo-Hookean energy, P, dP/dF; the
            Cauchy stress of Eq. 3/Eq. 4 (with the rest-state correction).
  mesh      rest shape, boundary-face extraction with parent tets
            (Algorithm 1, first three steps), contact band, vertex/face
            incidence, exact pixel binning.
  geometry  point-triangle / edge-edge distances and their derivatives, the
            IPC log barrier and edge-edge mollifier.
  ccd       additive continuous collision detection (conservative TOI).
  friction  IPC lagged friction (Sec. III-B's friction ratio and velocity
            threshold): lagged pairs, smoothed potential and derivatives.
  sim       the scene: incremental potential, Newton with a sparse direct
            solve, CCD-bounded backtracking line search, indenter substeps,
            stress / traction / pressure map / contact force (Algorithm 2),
            Algorithm 2's per-vertex force decomposition, the depth map of the
            deformed contact surface, per-tet materials.

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, invariants, finite differences or brute force.  The paper's own
outputs cannot pin anything (its figures are not available as numbers), so
agreement with the paper's printed results is "parity unpinned".
"""
