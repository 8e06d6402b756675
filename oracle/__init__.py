"""CPU oracle for FINOM (fast Sinkhorn for W1 on non-uniform meshes).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` and ``--impl reference`` legs) may import,
call, link or execute anything in this package.  The CUDA library in
``paper_2605_26659_gb300`` never routes through it; the two share no code.

Modules
-------
dense         plain dense float64 Sinkhorn (the definition; Sec. 2.1, eq.
              iteration, Algorithm 1 control flow), kernel products and cost.
finom_serial  the paper's dividing index, vector representations and p/q
              recurrences (Sec. 2.2-2.3, Algorithm 1, Remark on log-domain
              stabilisation, Algorithm 2 with Appendix A), pure Python.
exact         LP, 1D closed form W1 = int |F_mu - F_nu|, 2 x 2 entropic plan.
serial_c      the same recurrences in plain C for full-size inputs.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against values that do not come from the function itself (the paper's worked
example, LP optima, closed forms, invariants, brute force on tiny inputs).
"""
