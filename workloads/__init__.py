"""Seeded synthetic inputs for the multilayer quasi-periodic scattering solver.

This package only *describes* problems (interface shapes, layer wavenumbers,
incidence angles and discretisation sizes).  It holds none of the method's
arithmetic: both the CPU oracle (``oracle/``) and the CUDA path read the same
problem descriptions from here.
"""
from .problems import (Interface, PolyInterface, Params, Problem, config1, config2,
                       config3, config4, config5, corner_stack, flat_stack, small_stack,
                       trapezoid, wood_angle, CONFIGS)

__all__ = ["Interface", "PolyInterface", "Params", "Problem", "config1", "config2",
           "config3", "config4", "config5", "corner_stack", "flat_stack", "small_stack",
           "trapezoid", "wood_angle", "CONFIGS"]
