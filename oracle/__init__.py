"""FP64 CPU oracle of the VIP fractional-step method (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline/reference legs
may import this package.  The product path never does.
"""
