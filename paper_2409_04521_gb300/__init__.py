"""GB300-native adaptive ray-tracing radiative-transfer step of FlexRT
(Cain & D'Aloisio, arXiv:2409.04521).

The method runs in the CUDA kernels of ``libflexrt.so`` (sources in
``csrc/``, C ABI in ``include/flexrt.h``); ``flexrt`` is its ctypes binding.
"""
from .flexrt import (Batch, FlexRTError, Simulation, default_options, lib, library_path, probe_direction,  # noqa: F401
                     probe_merge, probe_merge_pixel, probe_pixvec, probe_rates, probe_rotation, probe_traverse)
