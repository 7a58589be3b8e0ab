"""Plain CPU oracle for the Census Template Matching path.

TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the CUDA library package.
"""
