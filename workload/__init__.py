"""Seeded synthetic inputs for the Hubbard exact-diagonalization hot path.

This package holds only input recipes: lattice bond lists, seeded start
vectors and seeded request lists.  It contains none of the method's
arithmetic (no basis, ranking, signs, H*v or Lanczos), so both the CPU
oracle and the CUDA path may draw their inputs from it.
"""
from .lattices import ring, square, dimer, lattice_by_name
from .vectors import splitmix64, start_vector, start_vector_into, start_vector_at
from .requests import batch_sectors, serve_requests

__all__ = ["ring", "square", "dimer", "lattice_by_name", "splitmix64", "start_vector", "start_vector_into",
           "start_vector_at", "batch_sectors", "serve_requests"]
