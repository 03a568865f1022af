"""Plain FP64 CPU oracle for the STBA Levenberg-Marquardt iteration.

TEST INFRASTRUCTURE ONLY.  Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The product path (the CUDA library and its Python binding) never
imports it and shares no code with it.

It follows the paper ("Stochastic Bundle Adjustment for Efficient and Scalable 3D Reconstruction",
Zhou et al., ECCV 2020) step by step, in its notation, with SciPy sparse matrices standing for the
paper's matrices:
  camera.py  -- the reprojection error f of Sec. 3 and its Jacobian (complex-step differentiation);
  stba.py    -- the normal-equation blocks of Eq. 4, the Schur step of Eq. 5-6 (full-RCS LM), the
                clustered system of Eq. 10 with point splitting/binding (Sec. 4.1-4.2), the per-cluster
                solves of Eq. 13, the point update of Eq. 15, the steepest-descent correction of Sec. 4.3,
                and the LM control of Algorithm 1 (Appendix C), plus brute-force solvers for pins;
  sgc.py     -- stochastic graph clustering of Sec. 4.4 (modularity, Eq. 16 join probabilities, the
                sampler, and the exact distribution of final clusterings on tiny graphs);
  adjoint.py -- the reverse pass through K recorded iterations (not in the paper: implicit
                differentiation of each accepted step's damped, cluster-split normal equations).

Every function is pinned by `tests/test_oracle_*.py` against something other than itself: finite
differences, library rotations, brute-force dense solves of Eq. 3 and Eq. 9, closed forms and invariants.
"""
from . import camera, sgc, stba  # noqa: F401
