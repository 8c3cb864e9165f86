"""The inputs of the GPU regression test for tile neighbourhoods across a short
last tile are sensitive: on the 200 x 136 grid (column tiles of 64, the last
one 8 wide; bands of 32 rows, the last 8 high), the atoms in column 0 put more
than the test's tolerance into columns 189 .. 191 of column tile 2, and the
atoms in row 0 into rows 125 .. 127 of band 3 -- pixels two tiles over through
the periodic wrap, which a neighbourhood counted in whole tiles misses.
Computed with the oracle alone (CPU)."""

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("dz", [2.5, 2.0])
def test_short_last_tile_regression_inputs_are_sensitive(dz):
    g = O.Grid(200, 136, 40.0, 27.0, 3, dz, 0.5, 200.0, 2.0 / 3.0)
    rng = np.random.default_rng(31)
    n = 120
    x, y, z = rng.uniform(0.0, 40.0, n), rng.uniform(0.0, 27.0, n), rng.uniform(0.5, 0.5 + 3 * dz, n)
    x[:n // 2] = rng.uniform(0.0, 40.0 / 200, n // 2)
    y[n // 2:] = rng.uniform(0.0, 27.0 / 136, n - n // 2)
    pos = np.stack([x, y, z], axis=1).astype(np.float32).astype(np.float64)
    species = np.zeros(n, np.int32)
    amp_sigma = [[27.0, 0.41]]
    full = O.projected_potential(g, pos, species, amp_sigma)
    tol = 2e-6 * np.max(np.abs(full)) + 1e-6
    col0 = O.projected_potential(g, pos[:n // 2], species[:n // 2], amp_sigma)
    row0 = O.projected_potential(g, pos[n // 2:], species[n // 2:], amp_sigma)
    assert np.max(np.abs(col0[:, :, 189:192])) > 10 * tol       # column tile 2 (columns 128 .. 191)
    assert np.max(np.abs(row0[:, 125:128, :])) > 10 * tol       # band 3 (rows 96 .. 127)
