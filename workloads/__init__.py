"""Seeded synthetic snapshot streams shaped like the paper's workloads.

This package holds input generators only -- none of the decomposition's
arithmetic.  Both the CUDA path's tests/benchmarks and the CPU oracle read the
same generated arrays.  The paper's datasets (JHTDB channel flow, the
ignition run, NSTX GPI) are not available; these generators stand in for them
with the shapes, sizes and value ranges the paper describes (Sec. 4).
"""
from .synth import (config1_matrix, ChannelFlowStream, IgnitionStream,
                    ImagingStream, LowRankStream, batched_streams_spec)

__all__ = ["config1_matrix", "ChannelFlowStream", "IgnitionStream",
           "ImagingStream", "LowRankStream", "batched_streams_spec"]
