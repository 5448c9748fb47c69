"""GB300-native LSMS Kubo-Greenwood conductivity hot path (arXiv 2311.12134).

The compute path lives in the CUDA/C++ shared library ``liblsmskubo.so``
(sources in ``csrc/``, C ABI in ``include/lsmskubo.h``); ``binding`` marshals
arguments to it.  ``workload`` holds the seeded synthetic input generators.
The library is loaded on first use, so the generators import on machines
without the library; every compute call raises if the library is missing.
"""
from . import workload  # noqa: F401

__all__ = ["workload"]
