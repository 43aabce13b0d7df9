"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds only random-number generation and point sets; none of the
H^2 product's arithmetic lives here.
"""
from .points import splitmix64, uniform01, normal01, sphere, cube, cube_surface, cube_surface_normals, make_points

__all__ = ["splitmix64", "uniform01", "normal01", "sphere", "cube", "cube_surface", "cube_surface_normals",
           "make_points"]
