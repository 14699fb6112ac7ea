"""Host logic of the binding's two-stage multigrid autotuner (vip.autotune), on a
fake context (no GPU): stage 1 is vip_autotune's table of zero-guess solves; stage
2 re-runs only the `refine` fastest converged pairs for `refine_steps` steps from
the initial fields and keeps the one with the fewest Poisson iterations in the
warm-started steps; the state is reset afterwards and the choice is cached per
geometry signature."""
import numpy as np

import workloads as w
from paper_1401_6513_gb300 import vip


class FakeStats:
    def __init__(self, total):
        self.total_poisson_iters = total


class FakeCtx:
    """Zero-guess solve times and per-step iteration counts per (omega, corr)."""

    def __init__(self, ms, step_iters):
        self.ms, self.step_iters = ms, step_iters
        self.params = (1.0, 1.5)
        self.total = 0
        self.calls = []
        self.resets = 0

    def vip_step(self, n):
        self.calls.append(("step", n, self.params))
        self.total += n * self.step_iters[self.params]

    def vip_get_stats(self):
        return FakeStats(self.total)

    def vip_set_multigrid(self, omega, corr):
        self.params = (round(omega, 4), round(corr, 4))

    def vip_set_state(self, u, v, p):
        self.resets += 1

    def vip_autotune(self, omegas, corrs):
        pairs = [(o, c) for o in omegas for c in corrs]
        ms = self.ms

        class Result:
            def as_dict(self_inner):
                best = min((k for k in pairs if ms[k] >= 0), key=lambda k: ms[k])
                return {"omega": best[0], "corr": best[1],
                        "candidates": [{"omega": o, "corr": c, "iters": 10, "ms": ms[(o, c)]}
                                       for o, c in pairs]}
        return Result()


def make(ms_table, iters_table):
    return FakeCtx(ms_table, iters_table)


def test_refine_picks_fewest_warm_started_iterations(tmp_path):
    ns = w.cavity(8, Re=100.0)
    omegas, corrs = (0.9, 1.0), (1.5, 1.7, 1.9)
    # zero-guess times: (0.9, 1.7) fastest, then (1.0, 1.7), then (1.0, 1.9); (0.9, 1.9)
    # did not converge (ms < 0)
    ms = {(0.9, 1.5): 9.0, (0.9, 1.7): 5.0, (0.9, 1.9): -1.0,
          (1.0, 1.5): 8.0, (1.0, 1.7): 5.5, (1.0, 1.9): 6.0}
    # warm-started steps: (1.0, 1.7) needs the fewest iterations; (1.0, 1.5) would be
    # better still but is not among the three fastest
    iters = {(0.9, 1.5): 40, (0.9, 1.7): 70, (0.9, 1.9): 10,
             (1.0, 1.5): 30, (1.0, 1.7): 60, (1.0, 1.9): 65}
    ctx = make(ms, iters)
    cache = tmp_path / "tune.json"
    entry = vip.autotune(ctx, [ns], cache=cache, omegas=omegas, corrs=corrs, refine=3, refine_steps=3)
    assert (entry["omega"], entry["corr"]) == (1.0, 1.7)
    assert ctx.params == (1.0, 1.7)
    refined = [c for c in entry["candidates"] if "step_iters" in c]
    assert sorted((c["omega"], c["corr"]) for c in refined) == [(0.9, 1.7), (1.0, 1.7), (1.0, 1.9)]
    # each re-run: one step from the initial fields, then two scored steps
    assert {c["step_iters"] for c in refined} == {2 * 70, 2 * 60, 2 * 65}
    assert ctx.resets == 3 + 1  # before each re-run and once at the end
    assert not entry["cached"] and entry["refined_on_steps"] == 2
    # a second context with the same geometry takes the cached choice without tuning
    ctx2 = make(ms, iters)
    again = vip.autotune(ctx2, [ns], cache=cache, omegas=omegas, corrs=corrs)
    assert again["cached"] and (again["omega"], again["corr"]) == (1.0, 1.7)
    assert ctx2.calls == [] and ctx2.params == (1.0, 1.7)


def test_single_converged_pair_skips_refinement():
    ns = w.cavity(8, Re=100.0)
    ms = {(1.0, 1.5): 4.0, (1.0, 1.7): -1.0}
    ctx = make(ms, {(1.0, 1.5): 50, (1.0, 1.7): 5})
    entry = vip.autotune(ctx, [ns], omegas=(1.0,), corrs=(1.5, 1.7))
    assert (entry["omega"], entry["corr"]) == (1.0, 1.5)
    assert "refined_on_steps" not in entry
    assert [c for c in ctx.calls if c[0] == "step"] == [("step", 1, (1.0, 1.5))]


def test_geometry_signature_tracks_nodes():
    a, b = w.cavity(8, Re=100.0), w.cavity(9, Re=100.0)
    assert vip.geometry_signature([a]) == vip.geometry_signature([w.cavity(8, Re=400.0)])
    assert vip.geometry_signature([a]) != vip.geometry_signature([b])
    moved = w.cavity(8, Re=100.0)
    moved.x[3] += 1e-9
    assert vip.geometry_signature([moved]) != vip.geometry_signature([a])
    assert np.all(a.x == w.cavity(8, Re=100.0).x)


class ShiftCtx:
    """Fake context for choose_mg_shifts: Poisson iterations per node set for the
    context's cell-grid shifts; fails to step when told to."""

    def __init__(self, table, shifts, fail):
        self.table, self.shifts, self.fail = table, shifts, fail
        self.closed = False

    def vip_step(self, n):
        if self.fail:
            raise vip.VipError(vip.VIP_ERR_NOT_CONVERGED, "did not converge")

    def vip_get_geometry_iters(self):
        return np.array([self.table[g][s] for g, s in enumerate(self.shifts)], np.int64)

    def close(self):
        self.closed = True


def test_choose_mg_shifts_takes_each_geometry_s_fewest_iterations():
    a, b = w.cavity(8, Re=100.0), w.periodic_box(8)
    # per node set: iterations for each (shift_x, shift_y) the context was built with
    table = [{(0, 0): 90, (1, 0): 120, (0, 1): 40, (1, 1): 55},
             {(0, 0): 30}]                       # periodic: always (0, 0)
    made = []

    def make(nodesets, mg_shifts, **kw):
        assert kw == {"rtol": 1e-8}
        ctx = ShiftCtx(table, mg_shifts, fail=(mg_shifts[0] == (1, 1)))
        made.append((mg_shifts, ctx))
        return ctx

    shifts, its = vip.choose_mg_shifts([a, b], make=make, rtol=1e-8)
    assert shifts == [(0, 1), (0, 0)]
    assert [m[0] for m in made] == [[(0, 0), (0, 0)], [(1, 0), (0, 0)], [(0, 1), (0, 0)],
                                    [(1, 1), (0, 0)]]
    assert all(ctx.closed for _, ctx in made)
    # the failed context counts as the worst for both node sets
    assert its.shape == (4, 2) and its[3, 0] == its[3, 1] == np.iinfo(np.int64).max
    assert list(its[:3, 0]) == [90, 120, 40]


def test_cache_key_includes_the_cell_grid_parity(tmp_path):
    """A choice tuned on one cell-grid parity is not reused for another."""
    ns = w.cavity(8, Re=100.0)
    ms = {(1.0, 1.5): 4.0, (1.0, 1.7): 5.0}
    cache = tmp_path / "tune.json"
    plain = make(ms, {(1.0, 1.5): 50, (1.0, 1.7): 40})
    first = vip.autotune(plain, [ns], cache=cache, omegas=(1.0,), corrs=(1.5, 1.7))
    assert not first["cached"]
    shifted = make(ms, {(1.0, 1.5): 50, (1.0, 1.7): 40})
    shifted.mg_shift_key = lambda: "|mg:0:11"
    again = vip.autotune(shifted, [ns], cache=cache, omegas=(1.0,), corrs=(1.5, 1.7))
    assert not again["cached"] and shifted.calls
    third = make(ms, {})
    assert vip.autotune(third, [ns], cache=cache, omegas=(1.0,), corrs=(1.5, 1.7))["cached"]


def test_choose_mg_shifts_builds_each_distinct_assignment_once():
    boxes = [w.periodic_box(8), w.periodic_box(9)]
    made = []

    def make(nodesets, mg_shifts, **kw):
        made.append(mg_shifts)
        return ShiftCtx([{(0, 0): 12}, {(0, 0): 15}], mg_shifts, fail=False)

    shifts, its = vip.choose_mg_shifts(boxes, make=make)
    assert made == [[(0, 0), (0, 0)]]
    assert shifts == [(0, 0), (0, 0)] and (its == [[12, 15]] * 4).all()


class FakeFormCtx:
    """Per precision form: step time (ms) and whether its steps fail on the device."""

    def __init__(self, ms, failing=()):
        self.ms, self.failing = ms, set(failing)
        self.prec = None
        self.state = "initial"
        self.saved = None
        self.profiling = False
        self.steps_profiled = 0
        self.total = 0
        self.failed = False

    def vip_checkpoint(self, save, buf=None):
        if save:
            return ("ckpt", self.state)
        self.state = buf[1]
        self.failed = False
        return buf

    def vip_set_solver(self, prec, rtol, max_iters, identity):
        self.prec = prec

    def vip_step(self, n):
        self.state = ("stepped", self.prec)
        self.total += 10 * n
        if self.prec in self.failing:
            self.failed = True
        if self.profiling:
            self.steps_profiled += n

    def vip_get_stats(self):
        if self.failed:
            raise vip.VipError(vip.VIP_ERR_NONFINITE, "device reported status 6")
        return FakeStats(self.total)

    def vip_set_profiling(self, on):
        self.profiling = bool(on)
        if on:
            self.steps_profiled = 0

    def vip_get_profile(self):
        n = self.steps_profiled
        return {"rhs": 0.0, "poisson": self.ms[self.prec] * n}, n


def test_choose_precision_picks_fastest_form_and_restores_state():
    ctx = FakeFormCtx({vip.VIP_PREC_MIXED: 20.0, vip.VIP_PREC_FP64: 29.0, vip.VIP_PREC_MG32: 23.0})
    best, table = vip.choose_precision(ctx, candidates=(vip.VIP_PREC_FP64, vip.VIP_PREC_MIXED,
                                                        vip.VIP_PREC_MG32), steps=3)
    assert best == vip.VIP_PREC_MIXED and ctx.prec == vip.VIP_PREC_MIXED
    assert ctx.state == "initial"  # the caller continues from where it was
    assert [r["ms"] for r in table] == [29.0, 20.0, 23.0]


def test_choose_precision_skips_a_failing_form():
    ctx = FakeFormCtx({vip.VIP_PREC_MIXED: 90.0, vip.VIP_PREC_FP64: 74.0, vip.VIP_PREC_MG32: 10.0},
                      failing={vip.VIP_PREC_MG32})
    best, table = vip.choose_precision(ctx, candidates=(vip.VIP_PREC_MG32, vip.VIP_PREC_MIXED,
                                                        vip.VIP_PREC_FP64))
    assert best == vip.VIP_PREC_FP64
    assert table[0]["ms"] is None and "NONFINITE" in table[0]["error"]
    assert not ctx.profiling and ctx.state == "initial"


def test_choose_precision_raises_when_every_form_fails():
    ctx = FakeFormCtx({vip.VIP_PREC_MIXED: 1.0, vip.VIP_PREC_FP64: 1.0},
                      failing={vip.VIP_PREC_MIXED, vip.VIP_PREC_FP64})
    try:
        vip.choose_precision(ctx)
    except vip.VipError as e:
        assert e.status == vip.VIP_ERR_NOT_CONVERGED
    else:
        raise AssertionError("expected VipError")
    assert ctx.state == "initial"
