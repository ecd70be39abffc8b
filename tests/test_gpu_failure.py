"""Device-side failure detection of the tensor-core near field, without a GPU
fault: every mbarrier wait in that kernel is bounded; with the limit set to 0
polls every wait gives up at once, the kernel records the time-out in the
plan's device flag, frees its tensor memory and returns, and the host reports
LS_ERR_TIMEOUT.  Afterwards the context is still usable and the same plan gives
correct results again."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def plan():
    from paper_1509_05063_gb300 import Plan
    wl = W.place_cells(W.kite(n1=512, n2=17, h=0.025, kappa=6.0, collar_w=0.07, tau0=0.4, tau1=0.9, R_a=6,
                              R_b=5, R_cart=4, n_rho=32, N_tau=48), L=17, m=8, center=(-0.25, 0.0), N_eq=8)
    p = Plan(wl, W.n2_of(wl))
    yield p
    p.close()


def test_timeout_is_reported_and_recovered(plan):
    from paper_1509_05063_gb300 import LS_MIXED, LSError
    U = torch.from_numpy(W.random_density(plan.N, nrhs=16, seed=W.SEED + 31)).to("cuda:0", torch.complex64)
    good = plan.apply(U, prec=LS_MIXED)
    plan.device_status()                                   # nothing recorded
    plan.set_wait_limit(0)
    try:
        plan.apply(U, prec=LS_MIXED)
        with pytest.raises(LSError) as e:
            plan.device_status()
        assert e.value.status == 5
        plan.device_status()                               # the flag was cleared
        ui = torch.from_numpy(np.stack([W.plane_wave(plan.kappa, (1.0, 0.0), plan.nodes()[0])] * 16))
        with pytest.raises(LSError) as e:
            plan.solve(ui.to("cuda:0"), tol=1e-8, prec=LS_MIXED, max_iter=5)
        assert e.value.status == 5
    finally:
        plan.set_wait_limit(1 << 22)
    again = plan.apply(U, prec=LS_MIXED)
    plan.device_status()
    assert torch.equal(again, good)


def test_timeout_after_mmas_were_issued(plan):
    """Small non-zero limits: waits give up part-way through, after some bulk
    copies landed and some MMAs were issued (which limit does that depends on
    timing, so several are tried).  Each apply either completes or reports
    LS_ERR_TIMEOUT; the block always waits for its own MMAs and copies before
    it frees its tensor memory, so the next apply with the normal limit is
    exact again."""
    from paper_1509_05063_gb300 import LS_MIXED, LSError
    U = torch.from_numpy(W.random_density(plan.N, nrhs=16, seed=W.SEED + 32)).to("cuda:0", torch.complex64)
    good = plan.apply(U, prec=LS_MIXED)
    plan.device_status()
    timeouts = 0
    try:
        for limit in (1, 2, 4, 16, 64, 256, 1024, 4096):
            plan.set_wait_limit(limit)
            for _ in range(3):
                got = plan.apply(U, prec=LS_MIXED)
                try:
                    plan.device_status()
                    assert torch.equal(got, good)      # no time-out: the full result
                except LSError as e:
                    assert e.status == 5
                    timeouts += 1
    finally:
        plan.set_wait_limit(1 << 22)
    assert timeouts > 0
    again = plan.apply(U, prec=LS_MIXED)
    plan.device_status()
    assert torch.equal(again, good)
