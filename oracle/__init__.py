"""FP64 CPU oracle for the phase-field DUGKS step (arXiv:1810.07802, Sec. II).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline leg.  The product path never imports it.
"""
