"""Early ray termination on the GPU (Sec. 4): the running optical depth of a ray is
compared with tau_stop after each segment, and a ray that passes it adds nothing.

The kernel decides on its fp32 running sum, the oracle on the FP64 total. The two can
differ only for rays whose optical depth lies within rounding of tau_stop, and such a
ray changes a sink's flux by at most exp(-tau_stop) times its unabsorbed contribution.
So every sink must match the oracle to the usual tolerance, or differ from it by no
more than exp(-tau_stop) F(alpha = 0), on at most a few sinks."""
import numpy as np
import pytest

import workloads
from _parity import MAX_TOL, MEDIAN_TOL, gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu


def _check(f, of, f0, tau_stop, label, max_odd=2):
    f = np.asarray(f, np.float64)
    rel = np.abs(f - of) / np.maximum(of, 1e-300)
    ok = (rel <= MAX_TOL) | ((of < 1e-30) & (f < 1e-29))
    odd = np.nonzero(~ok)[0]
    assert len(odd) <= max_odd, f"{label}: {len(odd)} sinks off"
    assert np.all(np.abs(f[odd] - of[odd]) <= np.exp(-tau_stop) * f0[odd] * 1.01), label
    big = of >= 1e-30
    assert np.median(rel[big]) <= MEDIAN_TOL, label


def test_single_source_cutoff_gpu():
    from paper_1902_08083_gb300 import trevr
    P = workloads.stromgren(n_gas=1 << 16, alpha=20.0)
    G = gpu_tree(P)
    f, st = trevr.compute_flux(G, 0.75, 0.1, tau_stop=4.0, stats=True)
    f = f.cpu().numpy().astype(np.float64)
    s = np.linalg.norm(P["gas_xyz"].astype(np.float64) - 0.5, axis=0)
    ref = np.exp(-20.0 * s) / (4 * np.pi * s * s)
    cut = 20.0 * s > 4.0
    clear = np.abs(20.0 * s - 4.0) > 1e-3
    np.testing.assert_allclose(f[~cut & clear], ref[~cut & clear], rtol=1e-4)
    assert np.all(f[cut & clear] == 0.0)
    n_cut = int(np.count_nonzero(cut))
    assert abs(st["rays_terminated"] - n_cut) <= np.count_nonzero(~clear)


@pytest.mark.parametrize("tau_stop", [1.5, 4.0])
def test_termination_parity(tau_stop):
    from paper_1902_08083_gb300 import trevr
    P = workloads.uniform_box(n_gas=1 << 15, n_src=512, seed=40)
    rng = np.random.default_rng(41)
    P["alpha"] = workloads.lognormal_alpha(rng, P["gas_xyz"], 6.0, 1.5, 0.08)
    G = gpu_tree(P)
    T = oracle_tree(P)
    T0 = oracle_tree(dict(P, alpha=np.zeros_like(P["alpha"])))
    sinks = workloads.sink_sample(1 << 15, 2048, seed=42)
    f, c, st = trevr.compute_flux(G, 0.6, 0.1, tau_stop=tau_stop, counters=True, stats=True)
    of, oc = T.flux_terminated(0.6, 0.1, tau_stop, sinks=sinks, with_counters=True)
    f0 = T0.flux(0.6, 0.1, sinks=sinks)
    _check(f.cpu().numpy()[sinks], of, f0, tau_stop, f"tau_stop={tau_stop}")
    c = c.cpu().numpy()[sinks]
    # the walk is the complete one: interactions and visited cells as the oracle's
    np.testing.assert_array_equal(c[:, 0], oc[:, 0])
    np.testing.assert_array_equal(c[:, 2], oc[:, 2])
    # cut rays trace fewer segments
    assert np.all(c[:, 1] <= oc[:, 1])
    # all sinks: terminated-ray totals agree but for rays at the threshold
    _, oc_all = T.flux_terminated(0.6, 0.1, tau_stop, with_counters=True)
    n_cut = int(oc_all[:, 4].sum())
    assert n_cut > 0
    assert abs(st["rays_terminated"] - n_cut) <= max(2, n_cut // 100000)
    assert st["interactions"] == int(oc_all[:, 0].sum())


def test_termination_with_background_gpu():
    from paper_1902_08083_gb300 import trevr
    P = workloads.background_shell(n_gas=1 << 14, n_bg=4000, radius=0.45, alpha=8.0)
    G = gpu_tree(P)
    T = oracle_tree(P)
    T0 = oracle_tree(dict(P, alpha=np.zeros_like(P["alpha"])))
    f = trevr.compute_flux(G, 0.6, 0.1, tau_stop=2.0, bg_radius=0.45).cpu().numpy()
    of = T.flux_terminated(0.6, 0.1, 2.0, bg_radius=0.45)
    f0 = T0.flux_background(0.6, 0.1, 0.45)
    _check(f, of, f0, 2.0, "background + tau_stop")


def test_termination_only_for_the_plain_flux():
    import torch
    from paper_1902_08083_gb300 import trevr
    P = workloads.uniform_box(n_gas=2000, n_src=50, seed=43)
    G = gpu_tree(P)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux_moments(G, 0.75, 0.1, tau_stop=2.0)
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux_backward(G, torch.ones(2000, device="cuda"), 0.75, 0.1, tau_stop=2.0)
    for bad in (-1.0, float("nan")):
        with pytest.raises(trevr.TrevrError):
            trevr.compute_flux(G, 0.75, 0.1, tau_stop=bad)
    B = trevr.Batch([G])
    with pytest.raises(trevr.TrevrError):
        B.run(theta=0.75, tau_ref=0.1, tau_stop=2.0)
    B.free()
