"""Every form of the step other than plain FP64 against the FP64 oracle, per field.

The forms:
  * MIXED: each solve of Eqs. (12)-(13) by iterative refinement, an FP32 BiCGSTAB
    (FP32 arithmetic, vectors and operator copies, FP32 V-cycle) on the correction
    equation under an FP64 residual;
  * MG32: FP64 BiCGSTAB whose multigrid V-cycle runs in FP32;
  * LEARNED: FP64 solves started from the warm-start network's guess, trained on
    the run's own solves;
  * FP64 itself at the production tolerance, for scale.

Every form stops each solve on the same test, ||b - A x||_2 <= 1e-8 ||b||_2 with the
FP64 operator, so a form differs from the oracle (both solves run to 1e-13) by
what a 1e-8 stop leaves in the solution, not by its arithmetic.  The step count of
each case is the FP64 parity test's.  Bars (relative L2 over all nodes of the
case): u and v 1e-6, p 1e-4; the pressure bar is wider because p accumulates the
increments phi of every step and phi is determined by the solve only up to its
residual times the conditioning of the Poisson operator (~1e4-1e6 on these
node sets).  Each form must also stay within 100x the FP64 form's own error at
the same tolerance, so that a form whose arithmetic loses digits cannot hide
behind the absolute bar.
"""
import numpy as np
import pytest

import workloads as w
from oracle import vip_oracle as vo

pytestmark = pytest.mark.gpu

BAR = {"u": 1e-6, "v": 1e-6, "p": 1e-4}
REL_TO_FP64 = 100.0
FLOOR = 1e-12  # FP64 errors at the level of rounding: the relative check needs a floor


def cases():
    return {
        "periodic16": ([w.periodic_box(16, Re=100.0, dt=1e-3)], 20),
        "cavity20": ([w.cavity(20, Re=1000.0)], 20),
        "channel": ([w.channel_body(1 / 8, ("circle", 0.5), Re=100.0, xlim=(-3, 5), ylim=(-2, 2))], 10),
        "bumpy": ([w.channel_body(1 / 16, ("sines", 1.0, [(0.05, 12), (0.02, 31)]), Re=200.0,
                                  xlim=(-2.5, 4), ylim=(-2, 2))], 5),
        "triangle": ([w.triangle_cavity(33, Re=300.0)], 10),
        "batch4": ([w.triangle_cavity(33, Re=300.0, name="triangle33"), w.cavity(20, Re=1000.0),
                    w.channel_body(1 / 8, ("circle", 0.5), Re=100.0, xlim=(-3, 5), ylim=(-2, 2)),
                    w.triangle_cavity(45, Re=800.0, name="triangle45")], 6),
    }


CASES = cases()


def oracle_state(nss, nsteps):
    us, vs, ps = [], [], []
    for ns in nss:
        fs = vo.FractionalStep(vo.Operators(ns), rtol=1e-13)
        for _ in range(nsteps):
            fs.step()
        us.append(fs.u)
        vs.append(fs.v)
        ps.append(fs.p)
    return {"u": np.concatenate(us), "v": np.concatenate(vs), "p": np.concatenate(ps)}


def run_form(vip, nss, nsteps, form):
    prec = {"FP64": vip.VIP_PREC_FP64, "MIXED": vip.VIP_PREC_MIXED, "MG32": vip.VIP_PREC_MG32,
            "LEARNED": vip.VIP_PREC_FP64}[form]
    ctx = vip.solver_for(nss, precision=prec, rtol=1e-8, max_iters=50000)
    try:
        if form == "LEARNED":
            # the first steps collect samples, then the network trained on them
            # supplies the guess of the remaining steps
            k = max(2, nsteps // 2)
            ctx.vip_ws_collect(True, k)
            ctx.vip_step(k)
            ctx.vip_ws_collect(False)
            cfg = ctx.vip_ws_train(epochs=6, lr=1e-3, seed=3)
            assert np.isfinite(cfg.final_loss)
            ctx.vip_ws_enable(True)
            ctx.vip_step(nsteps - k)
        else:
            ctx.vip_step(nsteps)
        st = ctx.vip_get_stats()
        assert st.status == 0, (form, st.status)
        assert st.poisson_relres <= 1e-8 and st.helm_relres <= 1e-8, (form, st.poisson_relres)
        u, v, p, _ = ctx.vip_get_state()
    finally:
        ctx.close()
    return {"u": u, "v": v, "p": p}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module", params=list(CASES))
def case(request, vip):
    nss, nsteps = CASES[request.param]
    ref = oracle_state(nss, nsteps)
    fp64 = run_form(vip, nss, nsteps, "FP64")
    e64 = {f: rel(fp64[f], ref[f]) for f in "uvp"}
    return request.param, nss, nsteps, ref, e64


def test_fp64_at_production_tolerance(case):
    name, nss, nsteps, ref, e64 = case
    for f in "uvp":
        assert e64[f] <= BAR[f], (name, f, e64[f])


@pytest.mark.parametrize("form", ["MIXED", "MG32", "LEARNED"])
def test_form_matches_oracle_per_field(case, vip, form):
    name, nss, nsteps, ref, e64 = case
    got = run_form(vip, nss, nsteps, form)
    for f in "uvp":
        e = rel(got[f], ref[f])
        assert e <= BAR[f], (name, form, f, e)
        assert e <= REL_TO_FP64 * max(e64[f], FLOOR), (name, form, f, e, e64[f])
