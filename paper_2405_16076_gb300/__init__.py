"""GB300-native single-pass online randomized interpolative decomposition.

The method of Li, Becker & Doostan (arXiv 2405.16076, Algorithm 3 with the
coefficient updates of Algorithms 4-7 and the NA-Hutch++ estimator of
Algorithm 8) as hand-written sm_103a CUDA behind the C ABI of include/rid.h.
``paper_2405_16076_gb300.rid`` is the ctypes binding.
"""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def build(verbose=False):
    from .build import build as _b
    return _b(verbose=verbose)


def load():
    from . import rid
    return rid
