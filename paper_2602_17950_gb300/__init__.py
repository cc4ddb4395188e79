"""GB300 (sm_103a) ground-state solver for rotating spin-orbit-coupled spin-1
Bose-Einstein condensates: preconditioned nonlinear conjugate gradient with
cascadic multigrid on a Fourier-spectral grid (arXiv 2602.17950).

The numerical work happens in the CUDA library libgpsoc.so (C ABI in
include/gpsoc.h); this package only marshals arguments (see `gpsoc`).
"""
from .gpsoc import (GPSOC_FP64, GPSOC_MIXED, GPSOC_STOP_DPHI, GPSOC_STOP_ENERGY, GPSOC_STOP_RES,
                    GpsocError, Problem, Server, library, status_name)

__all__ = ["Problem", "Server", "GpsocError", "library", "status_name", "GPSOC_FP64", "GPSOC_MIXED",
           "GPSOC_STOP_DPHI", "GPSOC_STOP_RES", "GPSOC_STOP_ENERGY"]
