"""CPU oracle for the exact-summation path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package. ``xsum_oracle`` is the Python big-integer
definition; ``c_oracle`` loads the plain-C version of the same definition for
arrays too large for Python integers.
"""
