"""Seeded synthetic inputs for the all-at-once backward-Euler problem (eq. 2).

This package builds the spatial operators and right-hand sides of the
workloads (1D heat, 2D heat, 1D advection-diffusion) from a published
counter-free generator (SplitMix64 + Box-Muller).  It holds no arithmetic of
the ParaDiag method itself: no Fourier transform, no shifted solve, no Krylov
step.  Both the CUDA path's tests/benchmark and the CPU oracle draw their
inputs from here.
"""
from .gen import (  # noqa: F401
    SplitMix64,
    Problem,
    heat1d_operator,
    advdiff1d_operator,
    advdiff1d_centred_operator,
    advdiff1d_centred,
    heat2d_axis_operator,
    heat1d_127x64,
    heat1d_1023x1024,
    heat2d_255x255x256,
    advdiff1d_4095x2048,
    heat1d_sine_modes,
    heat1d_forced,
    heat2d_smooth,
    advdiff1d_pulse,
    random_tridiag_problem,
    with_mass,
    build_rhs,
    by_name,
)
