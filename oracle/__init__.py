"""CPU oracle for the DDM-GNN hot path: TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of what the paper's method computes, used to
check the CUDA path.  Only the test-suite, the smoke check and the benchmark's
CPU-baseline leg may import it; the library never does, and it shares no code
with the CUDA path (inputs come from the separate ``synth`` generators).

Modules, in the order of the method:

* ``fem``       P1 Galerkin assembly of the Poisson-Dirichlet problem (Section II, Eqs. 1-2).
* ``partition`` recursive coordinate bisection, overlap layers, partition of
                unity, Nicolaides coarse space, local DSS graphs (Section II-A, Section III-B).
* ``dss``       Deep Statistical Solver forward pass (Section III-B, Eqs. 18-22).
* ``ddm``       two-level additive Schwarz with exact local solves (DDM-LU,
                Eq. 7) and with DSS local solves (DDM-GNN, Section III-A,
                Eqs. 13-16); preconditioned CG (Algorithm 1) and flexible CG.

Equations are numbered in the order the paper prints them (Eq. 1 the
Poisson problem, Eq. 7 the two-level preconditioner, Eqs. 8-9 the
fixed-point form, Eq. 11 the residual loss, Eqs. 13-16 the three DDM-GNN
steps, Eqs. 18-22 the DSS block and decoder, Eqs. 24-25 the data family).

Every function names the passage it follows.  Readings of points where the
paper is silent are stated where they are used.
"""
