"""CPU FP64 oracle for the reduced-space interior-point method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or
run anything in this package.  The CUDA path never calls it, and it never
calls the CUDA path; the two share no code (only the seeded data generator in
``paper_2301_04869_gb300.synth`` feeds both, as data).

Modules:
  opf     -- the two-stage OPF model (objective, state equation g, operational
             constraints h) and its derivatives in complex-matrix notation.
  kkt     -- condensation (Prop. 2.1/2.2), reduction (Prop. 2.3), the Schur
             complement of the block-angular condensed system (Prop. 2.4) and
             dense checkers for the augmented system (eq. (6)).
  ipm     -- the primal-dual interior-point iteration (§2.2) that drives them.

Parity status of each function is given in its docstring; the OPF optimum
values themselves are "parity unpinned" beyond the pins listed in ipm.py
(no solution is printed in the paper).
"""
