"""FP64 CPU oracle of the time-domain Teukolsky solver -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  The product path never does.
"""
