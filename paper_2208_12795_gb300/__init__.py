"""GB300 (sm_103a) particle hot path of the envelope-tracking EM-FEMPIC method.

Modules: `inputs` (seeded synthetic workloads), `build` (compiles the CUDA
library), `capi` (ctypes binding of include/fempic_env.h), `env` (torch
wrapper: device memory and streams).  Importing the package loads nothing;
the library is loaded on first use and its absence is an error.
"""
