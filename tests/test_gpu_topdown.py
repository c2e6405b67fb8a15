"""The top-down ray walk on the GPU (trevr_params.ray_walk = 1; Sec. 3.1.3, last
paragraph of "Refinement Criterion"; Sec. 4) against the oracle's top-down walk,
element by element on the same seeded inputs: fluxes within the parity tolerance
and per-sink counters equal (both sides take the decisions in the same fp32 steps),
from 4096 particles up to the benchmark's 2^22 with its occluder."""
import numpy as np
import pytest

import workloads
from _parity import assert_flux_parity, clumpy_problem, gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu


def _run(G, theta, tau_ref, sinks=None, counters=True):
    import torch
    from paper_1902_08083_gb300 import trevr
    sidx = None if sinks is None else torch.from_numpy(np.asarray(sinks, np.int64)).cuda()
    if not counters:
        return trevr.compute_flux(G, theta, tau_ref, sink_idx=sidx, ray_walk=1).cpu().numpy()
    f, c, st = trevr.compute_flux(G, theta, tau_ref, sink_idx=sidx, counters=True, stats=True,
                                  ray_walk=1)
    return f.cpu().numpy(), c.cpu().numpy(), st


def _lognormal(P, sigma=2.0, seed=1, corr=0.05):
    rng = np.random.default_rng(seed)
    P["alpha"] = workloads.lognormal_alpha(rng, P["gas_xyz"], 1.0, sigma, corr, n_modes=128)
    return P


def test_topdown_uniform_closed_form_one_segment():
    P = workloads.stromgren(n_gas=1 << 16, seed=1, tau_ref=0.1)
    f, c, st = _run(gpu_tree(P), P["theta"], 0.1)
    r = np.linalg.norm(P["gas_xyz"].astype(np.float64) - 0.5, axis=0)
    assert_flux_parity(f, np.exp(-20.0 * r) / (4 * np.pi * r * r), "uniform top-down")
    assert np.all(c[:, 0] == 1) and np.all(c[:, 1] == 1) and st["refine_expansions"] == 0


@pytest.mark.parametrize("theta,tau_ref", [(0.75, 0.1), (0.6, 0.01), (0.75, 0.0), (0.75, 1e6),
                                           (0.0, 0.3)])
def test_topdown_lognormal_matches_oracle(theta, tau_ref):
    P = _lognormal(workloads.uniform_box(n_gas=12000, n_src=200, seed=21))
    f, c, st = _run(gpu_tree(P), theta, tau_ref)
    ref, rc = oracle_tree(P).flux_topdown(theta, tau_ref, with_counters=True)
    assert_flux_parity(f, ref, f"top-down theta={theta} tau_ref={tau_ref}")
    mism = np.nonzero(np.any(c != rc, axis=1))[0]
    assert len(mism) <= max(1, len(f) // 1000), f"{len(mism)} sinks with other decisions"
    assert st["interactions"] == rc[:, 0].sum()


def test_topdown_full_refinement_equals_bottom_up():
    # at tau_ref = 0 both walks sum the same leaves (in another order): the same
    # interactions, segments and visited cells; the refinement counts differ, since
    # the top-down walk splits every cell below A while the bottom-up walk lists the
    # cells along the two paths without splitting them
    from paper_1902_08083_gb300 import trevr
    P = _lognormal(workloads.uniform_box(n_gas=20000, n_src=100, seed=23))
    G = gpu_tree(P)
    f_td, c_td, _ = _run(G, 0.75, 0.0)
    f_bu, c_bu = trevr.compute_flux(G, 0.75, 0.0, counters=True)
    np.testing.assert_array_equal(c_td[:, :3], c_bu.cpu().numpy()[:, :3])
    np.testing.assert_allclose(f_td, f_bu.cpu().numpy(), rtol=2e-6)


def test_topdown_rejects_other_options():
    from paper_1902_08083_gb300 import trevr
    P = workloads.uniform_box(n_gas=2000, n_src=16, seed=2)
    G = gpu_tree(P)
    for kw in (dict(tau_stop=5.0), dict(bg_radius=0.4), dict(ray_walk=2)):
        with pytest.raises(trevr.TrevrError) as ei:
            trevr.compute_flux(G, 0.75, 0.1, **dict(dict(ray_walk=1), **kw))
        assert ei.value.code == 1
    import torch
    with pytest.raises(trevr.TrevrError):
        trevr.compute_flux_backward(G, torch.ones(2000, device="cuda"), 0.75, 0.1, ray_walk=1)


def test_topdown_clumpy_full_size_sampled():
    # the benchmark's workload: every sink walked on the GPU in the launch shape the
    # benchmark times; a seeded sample and every sink inside the occluder vs the oracle
    P = clumpy_problem()
    G = gpu_tree(P)
    f = _run(G, P["theta"], P["tau_ref"], counters=False)
    assert np.all(np.isfinite(f)) and np.all(f >= 0)
    inside = np.nonzero(np.all((P["gas_xyz"] >= 0.45) & (P["gas_xyz"] <= 0.55), axis=0))[0]
    sinks = np.concatenate([workloads.sink_sample(P["gas_xyz"].shape[1], 1024), inside])
    T = oracle_tree(P)
    ref = T.flux_topdown(P["theta"], P["tau_ref"], sinks=sinks)
    assert_flux_parity(f[sinks], ref, "clumpy top-down")
    G.free()
