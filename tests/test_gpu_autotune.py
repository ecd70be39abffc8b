"""The kernel-variant autotuner (ls_plan_autotune) on the GPU: it picks among
apply variants that give the same result up to rounding, so a tuned plan must
reproduce an untuned plan of the same workload within the precision bounds
(FP64: 1e-12 relative, the rounding of a different column-pass tiling;
complex64: 1e-5 element-wise, the mixed bound), and its report must name a
valid choice with timed candidates."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _kite():
    return W.place_cells(W.kite(n1=512, n2=17, h=0.025, kappa=6.0, collar_w=0.07, tau0=0.4, tau1=0.9, R_a=6,
                                R_b=5, R_cart=4, n_rho=32, N_tau=48), L=17, m=8, center=(-0.25, 0.0), N_eq=8)


def test_autotuned_plan_reproduces_the_default_variants():
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED, Plan
    wl = _kite()
    ref, tuned = Plan(wl, W.n2_of(wl)), Plan(wl, W.n2_of(wl))
    rep = tuned.autotune(16)
    assert rep["nrhs"] == 16
    assert rep["conv_cols64"] in (1, 2, 4, 8) and rep["conv_cols32"] in (1, 2, 4, 8)
    assert rep["group32"] in (4, 8, 16) and rep["near_cuda32"] in (0, 1)
    assert rep["near_cuda32"] == 0 or rep["group32"] >= 8
    assert rep["local_cuda32"] in (0, 1) and (rep["local_cuda32"] == 0 or rep["group32"] >= 8)
    assert rep["proj_cuda32"] in (0, 1) and (rep["proj_cuda32"] == 0 or rep["group32"] >= 8)
    assert rep["fft_radix32"] in (4, 16)
    assert rep["n_candidates"] >= 4 + 9 + 2
    assert 0 < rep["ms64_best"] <= rep["ms64_default"] and 0 < rep["ms32_best"] <= rep["ms32_default"]
    U = W.random_density(ref.N, nrhs=16, seed=W.SEED + 7)
    u64 = torch.from_numpy(U[0]).to("cuda:0")
    a = ref.apply(u64, prec=LS_FP64).cpu().numpy()
    b = tuned.apply(u64, prec=LS_FP64).cpu().numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-12
    u32 = torch.from_numpy(U).to("cuda:0", torch.complex64)
    a = ref.apply(u32, prec=LS_MIXED).cpu().numpy()
    b = tuned.apply(u32, prec=LS_MIXED).cpu().numpy()
    assert np.max(np.abs(a - b)) < 1e-5 * np.max(np.abs(a))
    tuned.device_status()
    ref.close()
    tuned.close()


def test_autotune_rejects_bad_calls():
    from paper_1509_05063_gb300 import LSError, Plan
    wl = _kite()
    p = Plan(wl, W.n2_of(wl))
    with pytest.raises(LSError) as e:
        p.autotune(0)
    assert e.value.status == 1
    with pytest.raises(LSError):
        p.autotune(65)
    p.close()
