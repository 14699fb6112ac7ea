"""What the learned warm start gains over the previous-increment guess, on held-out
steps, through the C ABI.

Workloads: the circular cylinder at h = 1/32 (525k nodes, Re 100) and the
256 x 256 lid-driven cavity (Re 1000), the flows the warm start is trained on.
Each runs in two contexts from the same initial fields: one collects its own
Poisson solves for K steps after a warm-up past the impulsive start and is then
trained (vip_ws_train: least-squares extrapolation coefficient a, then the
network on what the extrapolation leaves); the twin takes the same steps with
the plain guess phi^n.  Both then take M further (held-out) steps; every solve
stops on the same FP64 residual, 1e-8.

Asserted, as measured on GB300 (training is deterministic: fixed seed, fixed-order
reductions): (1) on both flows the learned extrapolation alone (vip_ws_enable mode
2) needs fewer Poisson iterations than phi^n over the held-out steps and less
Poisson time (it costs one vector update): cylinder 180 -> 154 iterations, cavity
296 -> 252; (2) the network on top of it is no robust gain: on the cavity it has
measured between 3 % fewer and 1 % more iterations depending on rounding details of
the training (the order of its sums), so the test only bounds its cost there (at
most 5 % more than the extrapolation alone); on the cylinder it loses (154 -> ~200):
there its BF16 correction at the lattice nodes, though it lowers the training loss
(a lattice-Laplacian proxy of the residual), raises the residual of the MLS Poisson
operator; (3) every guess gives the same solution to the solver tolerance.  The
measured counts and times are printed.
"""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu

W, K, M, EPOCHS = 30, 40, 10, 8


def cases():
    h = 1.0 / 32
    return {"cylinder_h32": w.channel_body(h, ("circle", 0.5), Re=100.0, dt=0.2 * h),
            "cavity_256": w.cavity(256, Re=1000.0)}


def poisson_run(ctx, steps):
    s0 = ctx.vip_get_stats()
    ctx.vip_set_profiling(True)
    ctx.vip_step(steps)
    prof, n = ctx.vip_get_profile()
    ctx.vip_set_profiling(False)
    s1 = ctx.vip_get_stats()
    return s1.total_poisson_iters - s0.total_poisson_iters, prof["poisson"] / max(n, 1)


@pytest.mark.parametrize("name", list(cases()))
def test_learned_warm_start_gains_on_held_out_steps(vip, name):
    ns = cases()[name]
    mk = lambda: vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-8, max_iters=50000)  # noqa: E731
    ctx, twin = mk(), mk()
    for c in (ctx, twin):
        c.vip_set_multigrid(1.0, 1.8)
        c.vip_step(W)
    ctx.vip_ws_collect(True, K)
    ctx.vip_step(K)
    ctx.vip_ws_collect(False)
    twin.vip_step(K)
    cfg = ctx.vip_ws_train(epochs=EPOCHS, lr=1e-3, seed=11)
    a = ctx.vip_ws_extrapolation()
    assert a == cfg.extrap and -1.0 <= a <= 2.0
    ck_twin = twin.vip_checkpoint(True)
    ck = ctx.vip_checkpoint(True)
    res = {}
    # the plain guess, on the twin
    twin.vip_step(1)  # graph capture outside the measured steps
    twin.vip_checkpoint(False, ck_twin)
    res["previous"] = poisson_run(twin, M)
    u_prev = twin.vip_get_state()[0]
    for mode, label in ((2, "extrapolation"), (1, "extrapolation+network")):
        ctx.vip_ws_enable(mode)
        ctx.vip_checkpoint(False, ck)
        ctx.vip_step(1)
        ctx.vip_checkpoint(False, ck)
        res[label] = poisson_run(ctx, M)
        u = ctx.vip_get_state()[0]
        assert np.linalg.norm(u - u_prev) <= 1e-6 * np.linalg.norm(u_prev), label
    print(name, "a =", round(a, 3), "loss", round(cfg.first_loss, 4), "->", round(cfg.final_loss, 4),
          "extrapolation alone", round(cfg.base_loss, 4), "network kept", cfg.net_kept,
          {k: (v[0], round(v[1], 3)) for k, v in res.items()})
    it_prev, ms_prev = res["previous"]
    it_ex, ms_ex = res["extrapolation"]
    it_net, _ = res["extrapolation+network"]
    assert it_ex < it_prev, res
    assert ms_ex < ms_prev, res
    if name == "cavity_256":
        assert it_net <= 1.05 * it_ex, res   # the network costs at most a few percent
    else:
        assert it_net > it_ex, res           # the network loses over the extrapolation
    ctx.close()
    twin.close()


def test_network_gains_with_thousands_of_samples(vip):
    """The cavity (256 x 256, Re 1000) trained on 2,000 of its own solves (4 epochs)
    instead of 40: on the 40 held-out steps that follow, every guess from the same
    checkpoint, the network on top of the extrapolation keeps and needs fewer Poisson
    iterations than the extrapolation alone, which needs fewer than phi^n (measured on
    GB300: 915, 853, 828; with the last 40 solves only: 915, 860, 900).  The samples
    take 2.9 MB each on this lattice."""
    ns = cases()["cavity_256"]
    ctx = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-8, max_iters=50000)
    ctx.vip_set_multigrid(1.0, 1.8)
    ctx.vip_step(W)
    ctx.vip_ws_collect(True, 2000)
    ctx.vip_step(2000)
    ctx.vip_ws_collect(False)
    cfg = ctx.vip_ws_train(epochs=4, lr=1e-3, seed=11)
    assert cfg.net_kept == 1 and cfg.final_loss < cfg.base_loss
    ck = ctx.vip_checkpoint(True)
    res = {}
    for mode, label in ((0, "previous"), (2, "extrapolation"), (1, "extrapolation+network")):
        ctx.vip_ws_enable(mode)
        ctx.vip_checkpoint(False, ck)
        ctx.vip_step(1)
        ctx.vip_checkpoint(False, ck)
        res[label] = poisson_run(ctx, 40)
    print("cavity_256, 2000 samples:", {k: (v[0], round(v[1], 3)) for k, v in res.items()})
    assert res["extrapolation+network"][0] < res["extrapolation"][0] < res["previous"][0], res
    ctx.close()


def test_fit_window_fits_the_recent_flow(vip):
    """The h = 1/32 cylinder with 400 collected solves from step 30, the impulsive
    start's large increments among them: the extrapolation coefficient fitted on the
    last 40 samples (vip_ws_set_fit_window) differs from the all-sample fit and needs
    no more Poisson iterations over 20 held-out steps from one checkpoint (2,000
    samples: 335 against 440 iterations over 40 steps)."""
    ns = cases()["cylinder_h32"]
    ctx = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-8, max_iters=50000)
    ctx.vip_set_multigrid(1.0, 1.8)
    with pytest.raises(vip.VipError):
        ctx.vip_ws_set_fit_window(-1)
    ctx.vip_step(W)
    ctx.vip_ws_collect(True, 400)
    ctx.vip_step(400)
    ctx.vip_ws_collect(False)
    ck = ctx.vip_checkpoint(True)
    res = {}
    for window in (0, 40):
        ctx.vip_ws_set_fit_window(window)
        cfg = ctx.vip_ws_train(epochs=1, lr=1e-3, seed=11)
        ctx.vip_ws_enable(2)
        ctx.vip_checkpoint(False, ck)
        ctx.vip_step(1)
        ctx.vip_checkpoint(False, ck)
        res[window] = (cfg.extrap, poisson_run(ctx, 20)[0])
    print("cylinder_h32, 400 samples: (a, held-out iterations) by fit window", res)
    assert res[40][0] != res[0][0]
    assert res[40][1] <= res[0][1], res
    ctx.close()
