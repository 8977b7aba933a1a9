"""GB300 (sm_103a) solver for 2D multilayer quasi-periodic scattering by the
periodizing integral-equation scheme of Cho & Barnett (arXiv 1410.5003).

The compute path lives in libmlqp.so (csrc/, C ABI in include/mlqp.h); the
Python side (mlqp.py) only marshals arguments and provides torch buffers.
"""
from . import mlqp  # noqa: F401
