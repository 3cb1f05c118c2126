"""GB300-native matrix-based omnidirectional pressure integration.

The solver lives in the C-ABI library ``libosmodi.so`` (CUDA kernels for
sm_103a); ``paper_2311_16935_gb300.osmodi`` is its thin Python binding and
``paper_2311_16935_gb300.inputs`` the seeded synthetic-input generators.
Importing the package loads neither.
"""

__all__ = ["osmodi", "inputs"]
