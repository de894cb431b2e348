"""The vehicle-level loop on the library (through the C ABI) equals the same loop on the oracle, vehicle
for vehicle: every decision's colony, the road model and the ticks agree bit for bit, so trip times,
paths, decision and retry counts are identical."""
import numpy as np
import pytest

from paper_2010_14244_gb300 import vehsim as V
from paper_2010_14244_gb300 import workloads as W
from tests.vehsim_oracle import OracleBackend

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    from paper_2010_14244_gb300 import build, gmacop

    build.build()
    return gmacop


@pytest.mark.parametrize("flags,alpha", [(0, 1.0), (224, 1.0), (0, 1.5)])
def test_library_loop_equals_oracle_loop(gm, orc, flags, alpha):
    wl = W.city52()
    src, dst = V.fleet(wl.net.n_nodes, 60, seed=7)
    cfg = V.SimConfig(n_ants=16, n_iter=4, alpha=alpha, flags=flags, seed=11)
    ctx = gm.Context(0)
    try:
        got = V.VehicleSim(V.LibraryBackend(ctx, wl, flags), cfg).run(src, dst, keep_paths=True)
    finally:
        ctx.close()
    want = V.VehicleSim(OracleBackend(orc, wl, flags), cfg).run(src, dst, keep_paths=True)
    assert got.arrived == want.arrived == 60
    np.testing.assert_array_equal(got.trip_ms, want.trip_ms)
    assert got.path_edges == want.path_edges
    assert (got.decisions, got.retries, got.steps) == (want.decisions, want.retries, want.steps)


def test_table_rows_grow_with_the_fleet(gm):
    """The experiment's rows on the library: every vehicle arrives, and the mean trip does not fall as
    the fleet grows from 100 to 1500 vehicles (more vehicles, longer queues)."""
    ctx = gm.Context(0)
    try:
        rows = V.run_table(ctx, [100, 1500], V.SimConfig(n_ants=16, n_iter=4))
    finally:
        ctx.close()
    assert [r["arrived"] for r in rows] == [100, 1500]
    assert rows[1]["mean_trip_s"] >= rows[0]["mean_trip_s"]
