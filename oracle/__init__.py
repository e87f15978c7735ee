"""Plain CPU oracle of the RBSM per-fragment path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA library in
``paper_1711_07793_gb300`` and never imports it.
"""
