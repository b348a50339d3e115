"""Plain, slow CPU oracle for the phasor–PIC hot path (arXiv 2609.15043).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from this
package.  The product path (the CUDA library and its Python binding) never
imports it, and this package never imports the product path: the two share no
code, headers, tables or constant generators.  Inputs that both sides consume
(synthetic particle populations, configurations) come from
``paper_2609_15043_b300.workloads``, which holds none of the method's
arithmetic; the oracle receives them as plain arguments.

Every function restates the paper's definition in the most direct form
available: sparse direct solves (``scipy.sparse.linalg``) for the field
equations, dense complex solves (``numpy.linalg``) for the circuit, and
vectorised numpy for the particle step.  Floating point is FP64 everywhere
except the particle step, which is written once over a dtype parameter: the
float32 instantiation takes every integer decision (cell crossing, collision
test, process choice) in the precision the kernels use, with the same
operation order, and the float64 instantiation is the accuracy reference.

Modules
-------
constants     physical constants (the paper's Test 3 values of eps0, mu0)
grid          RZ node/cell geometry, turn node sets, volumes and face areas
fields        FV Poisson, FD Helmholtz, Gauss-law turn charge, unit fields,
              vacuum impedance, node fields for the gather
circuit       turn-resolved network, controller, relaxation, residuals, powers
philox        Philox4x32-10 counter-based generator (Salmon et al. 2011)
particles     cross sections, cylindrical Boris push, null-collision MCC,
              area-weighted deposition, per-particle weights, secondary
              emission of absorbed ions
control       stochastic weighted split-merge particle control
mlp           the learned proposal's network, summaries, gate and training
cell          one RF cell advanced step by step and period by period, with
              the retained circuit harmonics
verification  the paper's particle-free Tests 1-3 set up on this oracle

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
except the particle step as a whole, whose only pins are invariants (closed
form Boris gyration, null-collision statistics, charge conservation, energy
bookkeeping); the paper prints no particle-level numbers.
"""
