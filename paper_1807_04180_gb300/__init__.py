"""GB300-native additive overlapping DDM for the Helmholtz equation.

The compute path lives in a C-ABI CUDA library (``csrc/``, built for sm_103a);
``paper_1807_04180_gb300.ddm`` binds it with ctypes.  ``workloads`` draws the
seeded synthetic inputs.  Importing the package does not load the library.
"""
__all__ = ["workloads"]
