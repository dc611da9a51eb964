"""GB300-native simulation step of non-episodic neuroevolution in a large
multi-agent common-pool-resource grid world (Hamon, Nisioti, Moulin-Frier,
2023).  The compute runs in the CUDA library libecoevo.so behind a C ABI
(include/ecoevo.h); this package only marshals arguments to it.
"""
from .params import EcoParams, PRESETS, held  # noqa: F401

__all__ = ["EcoParams", "PRESETS", "held"]
