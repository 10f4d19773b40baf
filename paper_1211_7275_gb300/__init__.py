"""GB300 (sm_103a) engine for the explicit-Euler relaxation of the discretised 1D quenched
Edwards-Wilkinson equation (Ferrero, Bustingorry, Kolton, arXiv:1211.7275).

The compute path is the C-ABI library ``libqew.so`` (include/qew.h) built from ``csrc/``;
this package is its Python binding.
"""
from ._capi import FP32_SPLIT, FP64, NONE, RB_GAUSS_CATMULLROM, RB_GAUSS_LINEAR, RB_UNIFORM_CATMULLROM, RF_GAUSS_LINEAR, QewError, load  # noqa: F401
from .relax import Relaxation, disorder_values, measure_alu_peaks, philox_words  # noqa: F401


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)
