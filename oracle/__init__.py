"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline leg and ``--impl reference``) may import this package.  The product
package never imports it and shares no code with it.
"""
