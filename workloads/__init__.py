"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This package draws random numbers and assembles CSR patterns; it holds none
of the sparse matrix-vector arithmetic under test.
"""
from . import rng  # noqa: F401
from .generators import *  # noqa: F401,F403
