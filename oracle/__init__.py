"""CPU oracle for Vietoris-Rips barcodes over Z/2 (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package. The GPU library never uses it.
"""
