"""Seeded synthetic workloads for the real-space DFT+U Chebyshev-filtered subspace iteration.

This package only draws random numbers and lays out geometry: grids, atom positions,
pseudopotential-like parameters, a Gaussian-model local potential and random starting
orbitals.  It holds none of the method's arithmetic (no finite differences, no projector
tables, no filter, no Rayleigh-Ritz), so the CPU oracle and the CUDA path can both consume
exactly the same inputs without sharing any computation.
"""
from .synthetic import (  # noqa: F401
    HARTREE_EV, BOHR_PER_ANGSTROM, Atom, Workload,
    tiny, rutile, rutile_snapshot, rutile_trajectory, anatase_cell, rutile_cell, snapshot_batch,
    small_test_system,
    gaussian_potential, random_orbitals, displaced, scaled_grid_for,
)
