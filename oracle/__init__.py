"""Oracle for the steady-state solve of Nation, Johansson, Blencowe & Rimberg,
"Iterative solutions to the steady state density matrix for optomechanical
systems" (arXiv:1411.4356).

TEST INFRASTRUCTURE ONLY.  A plain, slow, obviously-correct FP64 CPU
restatement of what the paper computes: the Liouvillian of Eq. 1, 3 and 4,
the trace-augmented system of Eq. 5, the RCM reordering of Sec. III, the
ILUT preconditioner of Sec. II, restarted GMRES of Sec. IV, the steady state,
its observables and the adjoint gradient.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA library
(``paper_1411_4356_gb300``) and neither imports the other.

Modules: ``liouvillian`` (Eq. 1-5, bandwidth/profile), ``reorder_factor``
(RCM, ILUT, triangular sweeps; plain C in ``oracle_native.c``), ``gmres``
(restarted right-preconditioned GMRES), ``steady`` (dense and iterative steady
states, observables, adjoint gradients), ``nojump`` (the no-jump part
K rho + rho K^dag of Eq. 3 and its inverse, the second preconditioner of the
GPU path).

Every function is pinned by tests under ``tests/test_oracle_*.py`` to facts
fixed by the paper or by the mathematics (the NNZ printed in Fig. 1, closed
forms at g0 = 0 and E = 0, exact invariants under truncation, brute force).
"""
