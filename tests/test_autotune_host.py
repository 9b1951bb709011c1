"""Host checks of the single-solve autotuner's search (no GPU: the timing and
the solve are stand-ins, the tile table is the library's own).

* it times every tile variant the library offers at every z-chunk setting,
  z-chunks longer than the column excepted, and the balanced-grid settings
  (negative z-chunks) too;
* a setting the solve refuses (the paired-cell variants on the balanced grid)
  ends that variant's search without an error;
* it leaves the solve configured with the fastest setting it timed.
"""

import pytest

from paper_1510_05061_gb300 import autotune, hydro, inputs


class FakeSim:
    """Records configure() calls; refuses what the library refuses."""

    def __init__(self, prob):
        self.prob = prob
        self.stream = None
        self.v = self.z = None
        self.calls = []

    def configure(self, v, z):
        if v in hydro.PAIR_VARIANTS and z < 0:
            raise hydro.HydroError(hydro.HYDRO_ERR_INVALID_ARG, "hydro_set_zchunk")
        self.v, self.z = v, z
        self.calls.append((v, z))

    def run_steps(self, n):
        pass


@pytest.fixture(scope="module")
def lib():
    from paper_1510_05061_gb300 import build

    build.build()
    hydro.load()
    return hydro


def test_search_covers_variants_and_balanced_settings(lib, monkeypatch):
    prob, _ = inputs.rayleigh_taylor(8, nz=100, precision=inputs.FP32)
    sim = FakeSim(prob)
    monkeypatch.setattr(autotune, "sim_signature", lambda s: "host-test")
    # a cost with its minimum at variant 6 on the balanced grid over whole columns
    monkeypatch.setattr(autotune, "time_sim_steps",
                        lambda s, steps: 1.0 + 0.01 * s.v + (0.0 if s.z == -1 else 0.5) + (0.0 if s.v == 6 else 0.3))
    choice = autotune.tune_simulation(sim, zchunks=(16, 64, 128, -1, -64), use_cache=False)
    assert (choice["variant"], choice["zchunk"]) == (6, -1)
    assert (sim.v, sim.z) == (6, -1)                   # left configured with the choice
    timed = {(r["variant"], r["zchunk"]) for r in choice["table"]}
    variants = dict(hydro.sim_variants())
    for v in variants:
        assert (v, 16) in timed and (v, 64) in timed
        assert (v, 128) not in timed                   # longer than the 100-plane column
        if v in hydro.PAIR_VARIANTS:
            assert (v, -1) not in timed and (v, -64) not in timed
        else:
            assert (v, -1) in timed and (v, -64) in timed
    for r in choice["table"]:
        assert r["async_staging"] == (4 <= r["variant"] < 8)
        assert r["paired_cells"] == (r["variant"] in hydro.PAIR_VARIANTS)
