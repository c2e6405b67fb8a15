"""The perturbed-glass stand-in at the paper's size, 64^3 gas and 64^3 stars (Sec. 3.1,
Appendix A), on the GPU:
- parity with the oracle on sampled sinks;
- the cost and error behaviour the paper prints for the glass (Sec. 3.1.2, 3.1.3;
  values in tests/golden/glass_accuracy.txt): the ratio of rays per element between
  theta_open = 0.45 and 0.75, a smaller error at the smaller angle, and an RMS error
  against tau_ref = 1e-8 below tau_ref."""
import numpy as np
import pytest
import torch

import workloads
from _golden import glass_accuracy
from _parity import assert_flux_parity, gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glass():
    P = workloads.perturbed_glass(64)
    return P, gpu_tree(P)


def _rms(f, ref):
    return float(np.sqrt(np.mean(((f - ref) / ref) ** 2)))


def test_glass_parity(glass):
    from paper_1902_08083_gb300 import trevr
    P, G = glass
    sinks = workloads.sink_sample(P["gas_xyz"].shape[1], 64, seed=15)
    f = trevr.compute_flux(G, 0.75, 0.1).cpu().numpy()
    assert_flux_parity(f[sinks], oracle_tree(P).flux(0.75, 0.1, sinks=sinks), "glass 64^3")


def test_glass_cost_and_error(glass):
    from paper_1902_08083_gb300 import trevr
    P, G = glass
    gold = glass_accuracy()
    n = P["gas_xyz"].shape[1]
    sinks = workloads.sink_sample(n, 512, seed=16)
    sk = torch.from_numpy(sinks).cuda()
    f0 = trevr.compute_flux(G, 0.0, 0.1, sink_idx=sk).cpu().numpy().astype(np.float64)
    rays, err = {}, {}
    for th in (0.45, 0.75):
        f, st = trevr.compute_flux(G, th, 0.1, stats=True)
        rays[th] = st["interactions"] / n
        err[th] = _rms(f.cpu().numpy()[sinks].astype(np.float64), f0)
    printed = (gold[("theta", 0.45)]["rays_per_element"] /
               gold[("theta", 0.75)]["rays_per_element"])
    assert abs(rays[0.45] / rays[0.75] / printed - 1.0) < 0.3
    assert err[0.45] < err[0.75] < 0.1
    fr = trevr.compute_flux(G, 0.75, 1e-8).cpu().numpy().astype(np.float64)
    for tr in (0.01, 0.1, 1.0):
        f = trevr.compute_flux(G, 0.75, tr).cpu().numpy().astype(np.float64)
        assert _rms(f, fr) < tr
