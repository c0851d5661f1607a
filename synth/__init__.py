"""Seeded synthetic workloads for the OVRO-LWA narrowband imaging hot path.

This package only *generates inputs*: antenna layouts, 4+4-bit coarse-channel
voltages with optional injected tones, and the frequency axes that describe
them.  It holds none of the method's arithmetic (no unpacking, FFT,
correlation, gridding or detection), so that both the CPU oracle and the CUDA
path can be fed the same bytes without sharing any of the computation.
"""
from .workloads import (  # noqa: F401
    C_LIGHT,
    Burst,
    Config,
    CONFIGS,
    Tone,
    antenna_positions,
    coarse_centre_hz,
    fine_freqs_hz,
    generate,
    generate_parallel,
    make_config,
    pack_nibbles,
    pfb_prototype,
    substream,
    splitmix64,
    tone_amplitude,
)
