"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package builds *inputs* only: bond sector lists (charge, dimension),
matrix-product-operator (MPO) site tensors for the lattice Hamiltonians of the
paper's Section V, and seeded Gaussian block values.  It holds none of the
effective-Hamiltonian arithmetic (no contraction, no charge-rule enumeration of
blocks): the oracle and the GPU library each enumerate allowed blocks on their
own and ask this package for the values of one block at a time, keyed by its
sector tuple.
"""
from .sectors import (binomial_sectors, paper_model_sectors, electron_sectors,
                      spin_phys, electron_phys)
from .mpo import (MPO, pair_term_mpo, heisenberg_pairs, chain_pairs,
                  cylinder_pairs, cylinder_hops, triangular_hops, snake_index, spin_ops, electron_ops,
                  heisenberg_mpo, hubbard_mpo, bulk_window, compress_mpo)
from .fill import (gaussian_block, env_block, assemble_flat, HeffWorkload,
                   spin_heff_workload, electron_heff_workload, hubbard_lattice_window,
                   triangular_hubbard_window, lattice_window,
                   workload_by_name)

__all__ = [
    "binomial_sectors", "paper_model_sectors", "electron_sectors", "spin_phys",
    "electron_phys", "MPO", "pair_term_mpo", "heisenberg_pairs", "chain_pairs",
    "cylinder_pairs", "cylinder_hops", "triangular_hops", "snake_index", "spin_ops", "electron_ops", "heisenberg_mpo",
    "hubbard_mpo", "bulk_window", "compress_mpo", "gaussian_block", "env_block", "assemble_flat",
    "HeffWorkload", "spin_heff_workload", "electron_heff_workload", "hubbard_lattice_window",
    "triangular_hubbard_window", "lattice_window",
    "workload_by_name",
]
