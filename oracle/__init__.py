"""Scalar C oracle for S4-BP128-D4 coding and sorted-list intersection.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the
CPU-baseline leg of bench.py.  The product path never loads it.
"""
from .oracle import Oracle, build_oracle  # noqa: F401
