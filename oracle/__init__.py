"""FP64 CPU oracle for the filtered-MgNet radiative-transfer solver.

This package is TEST INFRASTRUCTURE. It is a plain, slow, readable restatement
of the paper's mathematics in NumPy/SciPy (float64), written to check the CUDA
library against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_2604_23265_gb300``) never imports it and shares no
code, table or constant generator with it; the two meet only through the seeded
input generators in ``paper_2604_23265_gb300.workloads``, which hold none of
the method's arithmetic.

Modules
-------
tfps    -- DOM quadrature and HG kernel (Sec. 2.1, Eq. hg, Eq. DORTE_2d),
           TFPS eigenbasis, traces, the linear system A alpha = b
           (Sec. 2.2, Eqs. 2DTFPS_continuity_cond / boundary_cond / linear_sys),
           per-cell diagonal blocks, reconstruction (Eq. 2DTFPS_sol).
krylov  -- right-preconditioned flexible GMRES with modified Gram-Schmidt plus
           one reorthogonalisation, dense LU reference solve.
atfps   -- ATFPS selection, interface bases, projections and the filtered
           loss (Sec. 2.3, Eq. def_V_delta, Eq. loss_delta); the compressed
           system, its solve and the layer reconstruction (Sec. 2.3.3-2.3.4,
           Eqs. 2DAdaptiveTFPS_linear_sys, 2DAdaptive_TFPS_layer1 / layer2).
mgnet   -- CoeffNet + MgNet V-cycle forward/backward and Adam (Sec. 3).

Parity status of each function is stated in its docstring; functions with no
independent pin say "parity unpinned".
"""
