"""GB300 (sm_103a) implementation of the nullspace / ESPIRiT-equivalent coil-sensitivity
estimator with the PISCO accelerations (Lobos, Chan & Haldar, arXiv 2302.13431).

The computation lives in the CUDA library behind the C ABI of include/pisco.h; `_binding`
marshals arguments to it and `estimator` wraps it for torch tensors.  `phantoms` generates
seeded synthetic inputs.
"""
from . import phantoms  # noqa: F401

__all__ = ["phantoms"]
