"""CPU FP64 oracle for the periodizing multilayer scattering scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package; the product path
(the CUDA library and its Python binding) never does.
"""
from . import mlqp_oracle  # noqa: F401
