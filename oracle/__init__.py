"""CPU FP64 oracle for the Newton-based mixed-precision CARE refinement.

TEST INFRASTRUCTURE ONLY.  Nothing in the library (``paper_2607_14742_b300``)
imports, links or calls this package; only ``tests/``, the smoke check in
``__graft_entry__.py`` and the CPU-baseline leg of ``bench.py`` do.  It shares
no code with the CUDA path: its only common dependency is the seeded input
module ``care_inputs``, which holds no solver arithmetic.

Everything here is plain NumPy/SciPy in float64, written for obviousness, not
speed.  The one exception is the inner precision u_s of Framework 1
(``inner="fp32"``), in which NLR-ADI and the correction LR-ADI run on float32 /
complex64 arrays, so that NumPy and LAPACK compute them in IEEE single
precision, as in the FP32 rows of Section 5.1.  The paper's future-work precisions
(``inner="bf16"`` / ``"fp16"``) are modelled as FP32 arithmetic whose stored
results are rounded to the narrow format (``oracle.lowrank.storage_rounding``):

``oracle.dense``    -- the CARE residual operator, a Bartels-Stewart Lyapunov
                       solver, Newton's method in the paper's correction form
                       (Section 2, Eq. (2.1)-(2.2)), the Hamiltonian
                       invariant-subspace solution, and the scalar closed form.
``oracle.lowrank``  -- the low-rank realisation of Section 4 (inner precision
                       FP64 or FP32): LR-ADI with
                       projection shifts and Sherman-Morrison-Woodbury feedback
                       handling, NLR-ADI, the residual factor decomposition
                       (Algorithm 1), the solution factor decomposition
                       (Algorithm 2), Framework 1, and the paper's Res metric.
``oracle.precond``  -- ILU(0) of the shifted matrix (A + p I)^T, the GMRES
                       preconditioner of Section 5.2 (Saad's IKJ elimination
                       on the pattern).

Pins (see ``tests/test_oracle_*.py``): scalar closed form, eigenvector-aligned
closed forms (dense and on analytic Laplacian modes at any n), Hamiltonian
subspace and library CARE/Lyapunov solvers, ILU(0)'s pattern identity and its
agreement with LU wherever elimination makes no fill, Lyapunov closed forms, the
factored-residual identity R = F M F^T, ||H||_F = ||R||_F, the SMW identity
against a dense inverse, Newton monotonicity/quadratic convergence and the
invariants X = X^T >= 0, A - B B^T X stable; Table 1 (Section 5.1): the FP64 rows'
Res level and counts, and the FP32 rows' behaviour at the conditioning threshold
(convergence at kappa_2(A) = 1e2 in the paper's number of refinement steps,
no convergence at 1e8).
Shift selection inside LR-ADI is
a heuristic whose path is not pinned; only the Lyapunov/CARE solutions it
produces are (parity unpinned for the shift sequence itself).
"""
