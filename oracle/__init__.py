"""Plain FP64 CPU oracle for one ADER-DG time step on a 3:1 spacetree mesh.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library in
``paper_1806_07984_gb300`` never calls into it and shares no code with it.

The oracle is written to be read against the paper (Charrier, Hazelwood,
Weinzierl, "Enclave Tasking for DG Methods on Dynamically Adaptive Meshes"):

* ``basis``   - Gauss-Legendre nodes, Lagrange basis, derivative, time and
                inter-grid matrices (the discretisation of Sec. 2.1).
* ``pde``     - the balance law of Eq. (1): Euler and linear acoustics fluxes
                and wave-speed estimates.
* ``ader``    - the three tasks of Eq. (4) and Algorithm 1: the Picard
                space-time predictor C_STP with the projections id|dc and
                id|T+dT, the Rusanov solve F_R, the corrector C_Corr, the
                Cauchy-Kowalevski predictor for linear PDEs, and the CFL rule.
* ``mesh``    - the adaptive 3^d spacetree of Sec. 2.3: leaves, faces,
                virtual-cell prolongation, accumulate-Riemann restriction,
                skeleton/enclave classification and remeshing.
* ``step``    - Algorithm 1 extended by the AMR tasks of Sec. 2.3.

Every floating-point quantity is numpy float64.  Nothing is blocked, fused or
reordered beyond the paper's three task loops.
"""
