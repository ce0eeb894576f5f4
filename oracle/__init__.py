"""CPU FP64 oracle for the dp-adaptive MTO hot path (Gupta, van Keulen, Langelaar, arXiv:1811.09821).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct restatement of what the
GPU path computes, written from the paper.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The CUDA library under
``paper_1811_09821_gb300/`` never imports it, and it imports nothing from there: the two share no code.
The only shared module is ``workloads`` (seeded synthetic inputs, no method arithmetic).

Everything is float64 numpy / scipy.  A library primitive (Gauss-Legendre rule, dense Cholesky,
sparse LU, sort) may serve as one step; there is no blocking, fusion or reordering beyond the
definitions cited in each function.

Modules
-------
basis       Gauss-Legendre and Gauss-Lobatto-Legendre nodes, 1D Lagrange bases (App. B, Table B).
element     D0, subcell stiffness K_s0, composite element stiffness K_e (Eqs. 2-3, App. B).
mesh        structured dp-mesh, minimum-rule conformity and the canonical DOF numbering.
solve       global assembly, direct / PCG solves (Eq. 1).
sensitivity compliance C = f^T u and dC/drho_s (self-adjoint form; paper silent on the formula).
indicators  Kelly analysis indicator (Eq. 9), density indicator (Sec. 3.2.2), QR-error (Eq. 14),
            and the dp map update (Sec. 3.3).
oc          textbook optimality-criteria design update (paper silent on the optimizer).

Every function is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py`` except where its
docstring says "parity unpinned".
"""
