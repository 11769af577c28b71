"""Seeded synthetic inputs (geometry, C, V, D) shared by the oracle and the tests.

This package holds no part of the exchange computation itself: it only draws
the workloads and lays them out in the canonical packed format.
"""
from .systems import System, config, CONFIG_NAMES, water_cluster, ice, perovskite, ang2bohr, full_range
from .blocks import generate, pair_list, Packed, pack_key, unpack_key

__all__ = ["System", "config", "CONFIG_NAMES", "water_cluster", "ice", "perovskite",
           "ang2bohr", "full_range", "generate", "pair_list", "Packed", "pack_key", "unpack_key"]
