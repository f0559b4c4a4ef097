"""Seeded synthetic conductor meshes (inputs only).

This package builds the panelled (triangle or hybrid triangle/rectangle) conductor surfaces, terminal tags, ports,
material constants and frequency lists that both the CUDA library and the CPU
oracle consume.  It contains geometry construction only: no panel integral,
no impedance, no topology of the PEEC graph and no solver arithmetic.
"""
from .shapes import Mesh, bar, two_bars, coils, package, package_crop, pop, crop_check, panel_edges  # noqa: F401
