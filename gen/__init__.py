"""Seeded synthetic inputs shared by the oracle and the CUDA solver."""
from .grids import *  # noqa: F401,F403
