"""CPU oracle for the filtered-Lanczos normal-mode solver.

Test infrastructure only: a plain, slow FP64 restatement of what the solver
computes, written from the paper and pinned by the tests against closed
forms and invariants. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product never does,
and it shares no code with the CUDA library.
"""
