"""Inner tolerances of the MIXED form per solve (vip_set_inner_tolerance) and the
Helmholtz solve's extrapolated initial guess, through the C ABI.

The Helmholtz solves start from u^n + (u*^n - u^{n-1}) once a step has been taken
(an O(dt^2) guess where u^n is O(dt)); every solve still stops on the same FP64
residual, so the guess changes iteration counts, not the solution: ten MIXED steps
on the channel meet the oracle's state to the bar of the form tests, and both
Helmholtz tolerances give the same state to the solver tolerance.  With the default
Helmholtz inner tolerance (1e-6) the Helmholtz solves need no more iterations than
with the Poisson one's (1e-4).
"""
import numpy as np
import pytest

import workloads as w
from oracle import vip_oracle as vo

pytestmark = pytest.mark.gpu


def channel():
    return w.channel_body(1 / 8, ("circle", 0.5), Re=100.0, xlim=(-3, 5), ylim=(-2, 2))


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_inner_tolerance_arguments(vip):
    ctx = vip.solver_for(channel(), precision=vip.VIP_PREC_MIXED)
    for which, val in (("POISSON", 0.0), ("POISSON", 1.0), ("HELM_U", -1e-3), ("LAPLACE", 1e-4)):
        with pytest.raises(vip.VipError):
            ctx.vip_set_inner_tolerance(which, val)
    ctx.vip_set_inner_tolerance("POISSON", 3e-5)
    ctx.vip_set_inner_tolerance("HELM_U", 1e-7)
    ctx.vip_step(2)
    assert ctx.vip_get_stats().status == 0
    ctx.close()


def test_guess_and_tolerances_keep_the_solution(vip):
    ns = channel()
    fs = vo.FractionalStep(vo.Operators(ns), rtol=1e-13)
    for _ in range(10):
        fs.step()
    states, helm_its = {}, {}
    for label, helm_tol in (("default", None), ("loose", 1e-4)):
        ctx = vip.solver_for(ns, precision=vip.VIP_PREC_MIXED, rtol=1e-8)
        if helm_tol is not None:
            ctx.vip_set_inner_tolerance("HELM_U", helm_tol)
        ctx.vip_step(10)
        st = ctx.vip_get_stats()
        assert st.status == 0 and st.helm_relres <= 1e-8
        helm_its[label] = st.total_helm_iters
        states[label] = ctx.vip_get_state()[:3]
        ctx.close()
        for a, b, f in zip(states[label], (fs.u, fs.v, fs.p), "uvp"):
            assert rel(a, b) <= (1e-6 if f != "p" else 1e-4), (label, f, rel(a, b))
    for a, b in zip(states["default"], states["loose"]):
        assert rel(a, b) <= 1e-6
    assert helm_its["default"] <= helm_its["loose"], helm_its
