"""Early ray termination (Sec. 4, proposed there): a ray whose optical depth sum
passes tau_stop is abandoned and adds nothing.

Pins: the closed form for one source in a uniform medium (every ray's optical depth
is alpha s, so the flux is cut off at s = tau_stop / alpha); the definition applied to
the oracle's own interaction list (the terminated flux is the sum of the rays with
tau <= tau_stop, and the count of cut rays is the count of the others); the error
bound 0 <= F - F_stop <= exp(-tau_stop) F(alpha = 0); and tau_stop -> infinity giving
the plain flux bit for bit."""
import numpy as np
import pytest

import workloads


def _tree(oracle_lib, P):
    return oracle_lib.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"],
                                 bucket=P["bucket"])


def test_single_source_uniform_cutoff(oracle_lib):
    # one source of L = 1 at the centre, alpha = 20: tau = 20 s along every ray
    P = workloads.stromgren(n_gas=4096, alpha=20.0)
    T = _tree(oracle_lib, P)
    tau_stop = 4.0
    f, cnt = T.flux_terminated(0.75, 0.1, tau_stop, with_counters=True)
    s = np.linalg.norm(P["gas_xyz"].astype(np.float64) - 0.5, axis=0)
    ref = np.exp(-20.0 * s) / (4 * np.pi * s * s)
    cut = 20.0 * s > tau_stop
    clear = np.abs(20.0 * s - tau_stop) > 1e-6
    assert np.any(cut & clear) and np.any(~cut & clear)
    np.testing.assert_allclose(f[~cut & clear], ref[~cut & clear], rtol=1e-9)
    assert np.all(f[cut & clear] == 0.0)
    np.testing.assert_array_equal(cnt[clear, 4], cut[clear].astype(np.int64))


def test_termination_is_the_definition_on_the_interaction_list(oracle_lib):
    P = workloads.uniform_box(n_gas=3000, n_src=300, seed=31, alpha=1.0)
    rng = np.random.default_rng(32)
    P["alpha"] = workloads.lognormal_alpha(rng, P["gas_xyz"], 6.0, 1.5, 0.08)
    T = _tree(oracle_lib, P)
    tau_stop = 3.0
    sinks = workloads.sink_sample(3000, 60, seed=33)
    f, cnt = T.flux_terminated(0.6, 0.1, tau_stop, sinks=sinks, with_counters=True)
    n_cut_total = 0
    for k, i in enumerate(sinks):
        it = T.interactions(int(i), 0.6, 0.1)
        keep = it["tau"] <= tau_stop
        n_cut_total += int(np.count_nonzero(~keep))
        np.testing.assert_allclose(f[k], it["flux"][keep].sum(), rtol=1e-12, atol=1e-300)
        assert cnt[k, 4] == np.count_nonzero(~keep)
        assert cnt[k, 0] == it["tau"].shape[0]
    assert n_cut_total > 0
    # the other counters are those of the complete walk
    _, c0, _ = T.flux(0.6, 0.1, sinks=sinks, with_counters=True)
    np.testing.assert_array_equal(cnt[:, :4], c0)


def test_error_bound_and_limits(oracle_lib):
    P = workloads.uniform_box(n_gas=4000, n_src=200, seed=34)
    rng = np.random.default_rng(35)
    P["alpha"] = workloads.lognormal_alpha(rng, P["gas_xyz"], 5.0, 2.0, 0.05)
    T = _tree(oracle_lib, P)
    P0 = dict(P, alpha=np.zeros_like(P["alpha"]))
    T0 = _tree(oracle_lib, P0)
    sinks = workloads.sink_sample(4000, 300, seed=36)
    F = T.flux(0.75, 0.1, sinks=sinks)
    F0 = T0.flux(0.75, 0.1, sinks=sinks)  # same walk, no absorption
    for tau_stop in (1.0, 3.0, 8.0):
        Fs = T.flux_terminated(0.75, 0.1, tau_stop, sinks=sinks)
        d = F - Fs
        assert np.all(d >= -1e-12 * F)
        assert np.all(d <= np.exp(-tau_stop) * F0 * (1 + 1e-12))
    Fs = T.flux_terminated(0.75, 0.1, 1e30, sinks=sinks)
    np.testing.assert_array_equal(Fs, F)


def test_termination_rejects_bad_thresholds(oracle_lib):
    P = workloads.uniform_box(n_gas=500, n_src=20, seed=37)
    T = _tree(oracle_lib, P)
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(oracle_lib.OracleError):
            T.flux_terminated(0.75, 0.1, bad)


def test_termination_with_background_sources(oracle_lib):
    # with both options, the terminated flux is the background flux minus the cut rays
    P = workloads.background_shell(n_gas=3000, n_bg=2000, radius=0.45, alpha=8.0)
    T = _tree(oracle_lib, P)
    Fb = T.flux_background(0.6, 0.1, 0.45)
    Fs, cnt = T.flux_terminated(0.6, 0.1, 2.0, bg_radius=0.45, with_counters=True)
    assert np.all(Fs <= Fb * (1 + 1e-12))
    assert cnt[:, 4].sum() > 0
    np.testing.assert_array_equal(T.flux_terminated(0.6, 0.1, 1e30, bg_radius=0.45), Fb)
