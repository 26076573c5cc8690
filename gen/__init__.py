"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

Holds problem data only (trees, supports, marginals, cost matrices); none of the
solver's arithmetic lives here.
"""
from .problems import *  # noqa: F401,F403
from .problems import TreeProblem, COST_DENSE, COST_SQEUCLID  # noqa: F401
