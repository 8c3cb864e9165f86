"""Seeded synthetic inputs for the TACAW hot path.

This package holds only input generation: crystals, harmonic-mode
trajectories and the named workload configurations.  It contains none of the
method's arithmetic (no potentials, no multislice, no spectra), so both the
FP64 oracle and the CUDA path may consume what it produces as plain data.
"""

from .trajectory import (  # noqa: F401
    Crystal,
    HarmonicModes,
    simple_cubic,
    fcc,
    draw_modes,
    classical_amplitudes,
    positions,
    TrajectorySynth,
    static_positions,
)
from .configs import (  # noqa: F401
    Workload,
    GridSpec,
    WORKLOADS,
    batching_jobs,
    build_inputs,
)
from .series import modulated_waves  # noqa: F401
