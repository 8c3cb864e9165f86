"""Named synthetic workloads with explicit seeds.

Each workload mirrors the size and structure of a run the paper reports
(its Si, hBN and Fe set-ups use 560^2 to 1000^2 grids, hundreds to thousands
of slices and thousands of snapshots at 4-25 fs), at sizes that fit this
project's test and benchmark budget:

* ``plain_small``  -- simple-cubic 8x8x8 cells, a = 4 A, 64^2 grid over 32 A,
  8 slices of 4 A, 100 keV, 256 snapshots at 5 fs, 3 modes (20/45/80 meV).
* ``paper_scale``  -- fcc 20x20x50 cells, a = 4.05 A (80 000 atoms), 512^2
  grid over 81 A, 101 slices of 2 A, 200 keV, 4096 snapshots at 5 fs,
  200 modes (5-100 meV) with 300 K classical amplitudes.
* ``differentiation`` -- fcc 10x10x25, 256^2 over 40.5 A, 50 slices of 2 A,
  200 keV, 1024 snapshots, 100 modes.

Every atom is an isotropic Gaussian with projected peak amplitude 20 V*A and
width 0.3 A.  Random numbers come from ``default_rng(seed)`` in the order
documented in ``build_inputs``.
"""

from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from .trajectory import (
    Crystal,
    HarmonicModes,
    classical_amplitudes,
    draw_modes,
    fcc,
    positions,
    simple_cubic,
)


@dataclass(frozen=True)
class GridSpec:
    """Simulation grid and beam.  Lengths in Angstrom, beam energy in keV.

    Slice s covers [z0 + s*dz, z0 + (s+1)*dz); the first slice extends to
    -inf and the last to +inf for the purpose of splitting atoms.
    ``bandlimit`` is the fraction of the Nyquist radius kept by the propagator.
    """

    nx: int
    ny: int
    lx: float
    ly: float
    n_slices: int
    dz: float
    z0: float
    kev: float
    bandlimit: float = 2.0 / 3.0


@dataclass(frozen=True)
class Workload:
    name: str
    lattice: str                    # "sc" or "fcc"
    ncell: tuple
    a: float
    mass_u: float
    grid: GridSpec
    n_t: int
    dt_fs: float
    n_modes: int
    seed: int
    amp_sigma: tuple = ((20.0, 0.3),)   # per species: (projected amplitude V*A, sigma A)
    mode_energies: tuple | None = None  # fixed energies (meV); None = draw U[e_lo, e_hi]
    e_lo: float = 5.0
    e_hi: float = 100.0
    n_lo: tuple = (-10, -10, -25)
    n_hi: tuple = (10, 10, 25)
    rms_amp: float | None = None        # equal amplitudes giving this RMS |u|
    temperature_K: float = 300.0        # for classical amplitudes
    extra: dict = field(default_factory=dict)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    @property
    def gps(self) -> int:
        """Grid points x slices x snapshots of one full run."""
        g = self.grid
        return g.nx * g.ny * g.n_slices * self.n_t


WORKLOADS = {
    "plain_small": Workload(
        name="plain_small", lattice="sc", ncell=(8, 8, 8), a=4.0, mass_u=26.98,
        grid=GridSpec(64, 64, 32.0, 32.0, 8, 4.0, 0.0, 100.0),
        n_t=256, dt_fs=5.0, n_modes=3, seed=0,
        mode_energies=(20.0, 45.0, 80.0), n_lo=(-4, -4, -4), n_hi=(5, 5, 5),
        rms_amp=0.05,
    ),
    "paper_scale": Workload(
        name="paper_scale", lattice="fcc", ncell=(20, 20, 50), a=4.05, mass_u=26.98,
        grid=GridSpec(512, 512, 81.0, 81.0, 101, 2.0, 0.0, 200.0),
        n_t=4096, dt_fs=5.0, n_modes=200, seed=1,
        n_lo=(-10, -10, -25), n_hi=(10, 10, 25),
    ),
    "differentiation": Workload(
        name="differentiation", lattice="fcc", ncell=(10, 10, 25), a=4.05, mass_u=26.98,
        grid=GridSpec(256, 256, 40.5, 40.5, 50, 2.0, 0.0, 200.0),
        n_t=1024, dt_fs=5.0, n_modes=100, seed=4,
        n_lo=(-5, -5, -12), n_hi=(5, 5, 12),
    ),
}


def batching_jobs(n_jobs=64, seed0=1000, sizes=(128, 256, 384, 512, 768), slices=(10, 150),
                  snapshots=(512, 4096), n_modes=40):
    """Uneven independent trajectories (one Workload per job, seed seed0 + j).

    Draw order from default_rng(seed): grid size N (uniform over `sizes`),
    slice count, snapshot count (uniform integers, inclusive bounds), number of
    species (1-3), then per species the amplitude U[10, 30] V*A and width
    U[0.25, 0.40] A.  The fcc cell keeps the 0.158203125 A pixel of the
    paper-scale grid (N / 25.6 cells of 4.05 A laterally), enough cells along z
    to fill the slices; species are assigned per site in ``build_inputs``.
    """
    jobs = []
    for j in range(n_jobs):
        seed = seed0 + j
        rng = np.random.default_rng(seed)
        n = int(rng.choice(sizes))
        n_s = int(rng.integers(slices[0], slices[1] + 1))
        n_t = int(rng.integers(snapshots[0], snapshots[1] + 1))
        n_sp = int(rng.integers(1, 4))
        amp = rng.uniform(10.0, 30.0, n_sp)
        sig = rng.uniform(0.25, 0.40, n_sp)
        cells = int(round(n / 25.6))
        cz = int(np.ceil(n_s * 2.0 / 4.05))
        lx = cells * 4.05
        jobs.append(Workload(
            name=f"batch_job_{j}", lattice="fcc", ncell=(cells, cells, cz), a=4.05, mass_u=26.98,
            grid=GridSpec(n, n, lx, lx, n_s, 2.0, 0.0, 200.0),
            n_t=n_t, dt_fs=5.0, n_modes=n_modes, seed=seed + 100000,
            amp_sigma=tuple((float(a), float(b)) for a, b in zip(amp, sig)),
            n_lo=(-cells, -cells, -cz), n_hi=(cells, cells, cz),
            extra={"n_species": n_sp},
        ))
    return jobs


@dataclass
class Inputs:
    workload: Workload
    crystal: Crystal
    modes: HarmonicModes
    species: np.ndarray          # (Na,) int32
    amp_sigma: np.ndarray        # (n_species, 2) float32

    def times(self, snapshots=None) -> np.ndarray:
        idx = np.arange(self.workload.n_t) if snapshots is None else np.asarray(snapshots)
        return idx.astype(np.float64) * self.workload.dt_fs

    def positions(self, snapshots=None, dtype=np.float32) -> np.ndarray:
        """(T, Na, 3) positions for the given snapshot indices (default: all)."""
        return positions(self.crystal, self.modes, self.times(snapshots), dtype=dtype)

    def synth(self, device):
        """A TrajectorySynth of this workload's trajectory on `device`:
        synth(t0, t1, out) gives the positions of snapshots t0 .. t1-1."""
        from .trajectory import TrajectorySynth
        return TrajectorySynth(self.crystal, self.modes, self.workload.dt_fs, device=device)


def build_inputs(w: Workload) -> Inputs:
    """Build the crystal and modes of a workload.

    Draw order from default_rng(w.seed): species per site (if several), mode
    energies (if not fixed), then wave-vector indices, polarisations and
    phases (see ``draw_modes``).
    """
    rng = np.random.default_rng(w.seed)
    maker = simple_cubic if w.lattice == "sc" else fcc
    n_species = int(w.extra.get("n_species", 1))
    crystal = maker(w.ncell, w.a, w.mass_u, n_species=n_species, rng=rng if n_species > 1 else None)
    if w.mode_energies is not None:
        energies = np.asarray(w.mode_energies, dtype=np.float64)
    else:
        energies = rng.uniform(w.e_lo, w.e_hi, size=w.n_modes)
    if w.rms_amp is not None:
        # RMS of |u| over atoms and time is sqrt(sum_j a_j^2 / 2).
        amps = np.full(energies.shape, w.rms_amp / np.sqrt(energies.shape[0] / 2.0))
    else:
        amps = classical_amplitudes(energies, w.mass_u, w.temperature_K)
    modes = draw_modes(rng, crystal.cell, energies, amps, w.n_lo, w.n_hi)
    amp_sigma = np.asarray(w.amp_sigma, dtype=np.float32).reshape(-1, 2)
    return Inputs(w, crystal, modes, crystal.species.copy(), amp_sigma)
