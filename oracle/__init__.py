"""TEST INFRASTRUCTURE ONLY: the CPU oracle of the 3DGS training hot path.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.
"""
