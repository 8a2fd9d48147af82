"""Measured FP64 pipe peak of the current GPU (the ALU roofline of the stencil kernels).

    python -m paper_2010_04868_gb300.peak

compiles fp64_peak.cu with nvcc for sm_103a and prints its JSON result.
"""
