"""Plain FP64 CPU oracle for the blended P2-P1 Stokes operators and solver.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the CPU
baseline legs of bench.py, never by the library.  It shares no code with the CUDA path.
"""
