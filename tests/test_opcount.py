"""The benchmark's algorithmic-flop tables against the oracle's op-counting instantiation
(no GPU): the per-unit counts must add up to the count of a whole RHS evaluation."""
import pytest

import bench


def _total(r):
    return r["add"] + r["mul"] + r["div"] + r["sqrt"]


@pytest.mark.parametrize("key", sorted(bench.OPS_2D))
def test_2d_tables_add_up_to_the_oracle_rhs(orc, key):
    weights, split = key
    iface, cell, speed, diff, _rk = bench.OPS_2D[key]
    nx, ny = 8, 6
    # the oracle evaluates nx + 1 (ny + 1) interfaces per line and the split fluxes of every
    # padded cell (n + 6 per line) of both sweeps
    want = (iface * ((nx + 1) * ny + nx * (ny + 1)) + cell * ((nx + 6) * ny + (ny + 6) * nx)
            + (speed + diff) * nx * ny)
    assert _total(orc.opcount_rhs(2, nx, ny, weights, split)) == want
    parts = orc.opcount_parts(2, weights, split)
    assert (parts["interface"], parts["cell_per_sweep"], parts["wavespeed_cell"]) == (iface, cell, speed)


def test_1d_cell_update(orc):
    parts = orc.opcount_parts(1)
    per_stage = parts["interface"] + parts["cell_per_sweep"] + parts["wavespeed_cell"] + parts["difference_cell_per_dir"]
    assert 3 * per_stage + 36.0 == bench.OPS_1D_CELL_UPDATE
    assert (parts["interface"], parts["cell_per_sweep"], parts["wavespeed_cell"],
            parts["difference_cell_per_dir"]) == bench.OPS_1D
    n = 16
    assert _total(orc.opcount_rhs(1, n)) == (parts["interface"] * (n + 1) + parts["cell_per_sweep"] * (n + 6)
                                            + (parts["wavespeed_cell"] + parts["difference_cell_per_dir"]) * n)
