"""Seeded synthetic bundle-adjustment scenes shared by the oracle tests, the GPU tests and the benchmark.

This package is input generation only.  It draws ground-truth cameras and points, decides which camera
sees which point, synthesises noisy pixel observations and perturbs the initial parameters.  It holds none
of the solver's arithmetic: observations are made with SciPy's rotation routines, not with the oracle's
or the CUDA path's camera code, so a noise-free scene also checks both of those projections from outside.
"""
from .generate import (Scene, CONFIGS, make_config, make_ring_scene, make_hemisphere_scene,
                       make_slam_scene, make_tiny_scene, cluster_by_azimuth, cluster_sequence,
                       cluster_contiguous, subscene)

__all__ = ["Scene", "CONFIGS", "make_config", "make_ring_scene", "make_hemisphere_scene",
           "make_slam_scene", "make_tiny_scene", "cluster_by_azimuth", "cluster_sequence",
           "cluster_contiguous", "subscene"]
