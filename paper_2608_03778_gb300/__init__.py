"""GB300-native DiffPower hot path: levelized SP/TR propagation, its adjoint,
bit-parallel simulation and hybrid calibration behind a C-ABI library.

Submodules are imported on use, so that the input generator (``netgen``) can be
used on machines without the CUDA library.
"""
