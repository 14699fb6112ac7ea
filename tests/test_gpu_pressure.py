"""The pressure forms other than the default (vip_set_pressure) against the
oracle's FractionalStep readings of the same name, through the C ABI:
KIM_MOIN (Eq. 12 with no pressure term in r^n, Eq. 15 as p^{n+1} = phi - (dt/2Re)
L phi) and INCREMENTAL_INTERIOR (the incremental form with the (dt/2Re) L phi
term of Eq. 15 at interior nodes only).

All-FP64 steps, both sides' solves run to 1e-13, relative L2 <= 1e-10 on u, v, p
(the bar of the other step parity tests): the lid-driven cavity, the channel with
the circular cylinder (an outlet, so no bordered row), and the 28.072 degree wedge
of Sec. 5 with its normal points kept inside.  Switching the form between steps
takes effect at the next step (the captured step graph is replaced), on both
sides the same way.
"""
import numpy as np
import pytest

import workloads as w
from oracle import vip_oracle as vo

pytestmark = pytest.mark.gpu

CASES = {
    "cavity20": (lambda: w.cavity(20, Re=1000.0), "normal"),
    "channel": (lambda: w.channel_body(1 / 8, ("circle", 0.5), Re=100.0, xlim=(-3, 5), ylim=(-2, 2)),
                "normal"),
    "wedge33": (lambda: w.wedge_cavity(33, Re=1.0, dt=1.6 / 32 ** 2), "inside"),
}


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("form", ["kim_moin", "incremental_interior"])
@pytest.mark.parametrize("name", list(CASES))
def test_form_matches_oracle(vip, name, form):
    make, probes = CASES[name]
    ns = make()
    ctx = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-13, probes=probes,
                         pressure=form)
    fs = vo.FractionalStep(vo.Operators(ns, probes=probes), rtol=1e-13, pressure=form)
    ctx.vip_step(8)
    assert ctx.vip_get_stats().status == 0
    for _ in range(8):
        fs.step()
    u, v, p, _ = ctx.vip_get_state()
    for a, b, f in ((u, fs.u, "u"), (v, fs.v, "v"), (p, fs.p, "p")):
        assert rel(a, b) <= 1e-10, (name, form, f, rel(a, b))
    ctx.close()


def test_switching_forms_between_steps(vip):
    ns = w.cavity(20, Re=400.0)
    ctx = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-13)
    fs = vo.FractionalStep(vo.Operators(ns), rtol=1e-13)
    ctx.vip_step(3)  # the incremental form, its step graph captured
    for _ in range(3):
        fs.step()
    ctx.vip_set_pressure(vip.VIP_PRESSURE_KIM_MOIN)
    fs.pressure = "kim_moin"
    ctx.vip_step(3)
    for _ in range(3):
        fs.step()
    ctx.vip_set_pressure(vip.VIP_PRESSURE_INCREMENTAL_INTERIOR)
    fs.pressure = "incremental_interior"
    ctx.vip_step(2)
    for _ in range(2):
        fs.step()
    ctx.vip_set_pressure(vip.VIP_PRESSURE_INCREMENTAL)
    fs.pressure = "incremental"
    ctx.vip_step(2)
    for _ in range(2):
        fs.step()
    u, v, p, _ = ctx.vip_get_state()
    for a, b, f in ((u, fs.u, "u"), (v, fs.v, "v"), (p, fs.p, "p")):
        assert rel(a, b) <= 1e-10, (f, rel(a, b))
    with pytest.raises(vip.VipError):
        ctx.vip_set_pressure(3)
    ctx.close()
