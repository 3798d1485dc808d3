"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle (no method arithmetic)."""
from .rng import SplitMix64
from .molecules import (Molecule, Shell, water, water_cluster, organic_cloud,
                        batched_set, workload, draw_basis_set)

__all__ = ["SplitMix64", "Molecule", "Shell", "water", "water_cluster", "organic_cloud",
           "batched_set", "workload", "draw_basis_set"]
