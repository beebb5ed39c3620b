"""Host logic of the autotuner (no GPU): it keeps the fastest candidate whose every shifted system
converged, never picks an unconverged one, and stops trying cluster-resident candidates once a solve
shows the grid does not split into cluster strips (the kernel's work counter stays zero)."""
import types

import pytest

from paper_1409_2556_gb300 import autotune as AT
from paper_1409_2556_gb300._lib import KC, KC_COUNT


class FakeEngine:
    """Stands in for Engine: the cost and convergence of a forward solve are functions of the options."""

    def __init__(self, cost, converged, cluster_ok=True):
        self.cost, self.converged, self.cluster_ok = cost, converged, cluster_ok
        self.opts, self.calls, self.last_stats = {}, [], None

    def load_problem(self, prob, **opts):
        self.opts.update(opts)

    def set_options(self, **opts):
        self.opts.update(opts)

    def forward(self, times, allow_unconverged=False):
        o = dict(self.opts)
        self.calls.append(o)
        work = [0] * KC_COUNT
        if o.get("mg_cluster", 1) == 1 and self.cluster_ok:
            work[KC["inner"]] = 1000
        n = 100
        self.last_stats = {"ms_total": self.cost(o), "n_shift_solves": n,
                           "n_converged": n if self.converged(o) else n - 1, "work": work}
        return None


def _prob(nx=64):
    return types.SimpleNamespace(nx=nx, ny=64, nz=1, src_cells=[0, 1], rec_cells=[2], times=[1.0, 2.0], Nz=16,
                                 groups=1, tol=1e-10)


GRID = {"mg_cluster": [1, 0], "mg_tile": [1, 2], "sweeps": [(1, 2), (2, 2)], "inner": [(4, 6), (8, 6)],
        "inner_relax": [1e-4, 1e-3], "mg_tma": [1]}


def test_picks_fastest_converged_candidate():
    AT._CACHE.clear()
    # cluster candidates are faster; V(1,2) with relaxation 1e-3 is the fastest but does not converge
    def cost(o):
        c = 100.0 if o["mg_cluster"] == 1 else 150.0
        c -= 5.0 if o["mg_pre"] == 1 else 0.0
        c -= 2.0 if o["inner_relax"] == 1e-3 else 0.0
        return c + (1.0 if o["inner_rounds"] == 8 else 0.0)
    conv = lambda o: not (o["mg_pre"] == 1 and o["inner_relax"] == 1e-3)
    eng = FakeEngine(cost, conv)
    best = AT.autotune(eng, _prob(), {"tol": 1e-10, "Nz": 16, "groups": 1}, grid=GRID)
    assert best["mg_cluster"] == 1
    assert (best["mg_pre"], best["inner_relax"]) in ((1, 1e-4), (2, 1e-3))
    assert cost(best) == min(cost(o) for o in eng.calls if conv(o))
    assert conv(best)


def test_cluster_candidates_skipped_when_grid_does_not_split():
    AT._CACHE.clear()
    eng = FakeEngine(lambda o: 10.0 if o["mg_cluster"] == 1 else 20.0, lambda o: True, cluster_ok=False)
    best = AT.autotune(eng, _prob(nx=48), {"tol": 1e-10, "Nz": 16, "groups": 1}, grid=GRID)
    assert best["mg_cluster"] == 0
    n_cluster_calls = sum(1 for o in eng.calls if o.get("mg_cluster") == 1)
    assert n_cluster_calls == 2          # one candidate (warm-up + timed run), then the cluster branch stops


def test_result_cached_per_problem_shape():
    AT._CACHE.clear()
    eng = FakeEngine(lambda o: 1.0, lambda o: True)
    AT.autotune(eng, _prob(), {"tol": 1e-10}, grid=GRID)
    n = len(eng.calls)
    AT.autotune(eng, _prob(), {"tol": 1e-10}, grid=GRID)
    assert len(eng.calls) == n           # second call: no solves


def test_inner_tolerance_candidates_scale_with_tol():
    """inner_tol_factor candidates are multiples of the outer tolerance; the looser one wins only
    while every shifted system still converges."""
    AT._CACHE.clear()
    grid = dict(GRID, inner_relax=[1e-2], inner_tol_factor=[0.01, 0.1])
    cost = lambda o: 100.0 - (10.0 if o["inner_tol"] > 5e-12 else 0.0) - (1.0 if o["mg_pre"] == 1 else 0.0)
    eng = FakeEngine(cost, lambda o: True)
    best = AT.autotune(eng, _prob(), {"tol": 1e-10, "Nz": 16, "groups": 1}, grid=grid)
    assert sorted({round(o["inner_tol"], 15) for o in eng.calls}) == [1e-12, 1e-11]
    assert abs(best["inner_tol"] - 1e-11) < 1e-20
    AT._CACHE.clear()
    eng = FakeEngine(cost, lambda o: o["inner_tol"] < 5e-12)    # the looser tolerance misses some systems
    best = AT.autotune(eng, _prob(), {"tol": 1e-10, "Nz": 16, "groups": 1}, grid=grid)
    assert abs(best["inner_tol"] - 1e-12) < 1e-20
