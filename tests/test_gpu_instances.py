"""Several (T, mu, window) instances on shared meshes (vertex reuse across temperatures and
chemical potentials, section "Workflow and structure").  Each instance's rate list and
transport coefficients must match the oracle run on that instance alone (its own window, T
and mu); the shared-vertex path must agree with the direct single-instance path."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2109_08547_gb300 import binding as B
from paper_2109_08547_gb300 import synthetic as SY
from _parity import COEFF_RTOL, compare_rates, gpu_rate_table, oracle_rate_table, rel_fro

pytestmark = pytest.mark.gpu

TENSORS = ("sigma", "sigmaS", "alpha_el", "kappa0_el", "alpha_ph", "kappa_ph")
UNION = (-0.45, 0.45)
# (T_K, mu_eV, window_lo_eV, window_hi_eV): uneven windows inside the mesh window
INSTANCES = [(300.0, 0.0, -0.3, 0.3), (180.0, 0.12, -0.18, 0.42), (460.0, -0.15, -0.45, 0.05)]


def _union_workload():
    return dataclasses.replace(SY.workload_cscl4(n=6), window=UNION)


@pytest.fixture(scope="module")
def batched():
    wl = _union_workload()
    ctx = B.Context(0)
    B.set_wannier_model(ctx, wl.model)
    B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
    rates = B.compute_transition_rates(ctx, 0.0, 0.0, wl.sigma_eV, wl.cutoff_sigmas, instances=INSTANCES)
    solve = B.solve_coupled_bte(ctx, "dragged", wl.tol)
    coeffs = [B.transport_coefficients(ctx, i) for i in range(len(INSTANCES))]
    yield {"ctx": ctx, "wl": wl, "rates": rates, "solve": solve, "coeffs": coeffs}
    ctx.close()


@pytest.fixture(scope="module")
def standalone():
    """The oracle on each instance alone: its window is the mesh window."""
    out = []
    for T, mu, lo, hi in INSTANCES:
        w1 = dataclasses.replace(_union_workload(), T_K=T, mu_eV=mu, window=(lo, hi))
        P = O.prepare(w1)
        R = O.transition_rates(P)
        out.append((w1, P, R, O.solve_coupled_bte(P, R, level="dragged", ko=True)))
    return out


def test_instance_count_and_range(batched):
    ctx = batched["ctx"]
    assert B.num_instances(ctx) == len(INSTANCES)
    with pytest.raises(B.EphbError):
        B.select_instance(ctx, len(INSTANCES))
    with pytest.raises(B.EphbError):
        B.transport_coefficients(ctx, -1)


def test_instance_rates_match_oracle(batched, standalone):
    ctx, wl = batched["ctx"], batched["wl"]
    for i, (w1, P, R, _) in enumerate(standalone):
        B.select_instance(ctx, i)
        compare_rates(gpu_rate_table(ctx, wl), oracle_rate_table(R), P)


def test_instance_coefficients_match_oracle(batched, standalone):
    ctx = batched["ctx"]
    assert batched["solve"]["converged"] == 1
    for i, (_, _, _, ref) in enumerate(standalone):
        assert ref.converged
        info = B.instance_solve_info(ctx, i)
        assert info["converged"] == 1 and info["outer_iters"] >= 1
        for key in TENSORS:
            err = rel_fro(batched["coeffs"][i][key], ref.coeffs[key])
            assert err <= COEFF_RTOL, f"instance {i} {key}: {err:.3e}"


def test_solve_summary_adds_instances(batched):
    ctx, s = batched["ctx"], batched["solve"]
    infos = [B.instance_solve_info(ctx, i) for i in range(len(INSTANCES))]
    assert s["n_sweeps"] == sum(x["n_sweeps"] for x in infos)
    assert s["outer_iters"] == max(x["outer_iters"] for x in infos)
    assert s["n_runs"] == sum(x["n_runs"] for x in infos)


def test_shared_vertex_equals_direct_path():
    """One instance on the mesh window computed directly, and twice through the shared vertex:
    same rates (to rounding) and coefficients."""
    wl = SY.workload_cscl4(n=6)
    with B.Context(0) as c1, B.Context(0) as c2:
        for c in (c1, c2):
            B.set_wannier_model(c, wl.model)
            B.build_meshes_ibz(c, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
        B.compute_transition_rates(c1, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas)
        r2 = B.compute_transition_rates(c2, 0.0, 0.0, wl.sigma_eV, wl.cutoff_sigmas,
                                        instances=[(wl.T_K, wl.mu_eV), (wl.T_K, wl.mu_eV)])
        assert r2["n_entries"] == B.get_array(c2, "row_ptr")[-1]
        t1 = gpu_rate_table(c1, wl)
        for i in (0, 1):
            B.select_instance(c2, i)
            t2 = gpu_rate_table(c2, wl)
            assert set(t1) == set(t2)
            a = np.array([t1[k] for k in t1])
            b = np.array([t2[k] for k in t1])
            assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))
        B.solve_coupled_bte(c1, "dragged", wl.tol)
        B.solve_coupled_bte(c2, "dragged", wl.tol)
        g1 = B.transport_coefficients(c1)
        for i in (0, 1):
            g2 = B.transport_coefficients(c2, i)
            for key in TENSORS:
                assert rel_fro(g2[key], g1[key]) <= 1e-10, key


def test_deferred_instances_give_the_same_answers(batched, standalone):
    """Instances whose lists are derived only when the solve reaches them (what the library does
    when all instances' lists would not fit the device memory; forced here): every instance's
    coefficients bit-identical to the eagerly derived ones and within 1e-8 of the oracle on the
    instance alone; a second solve (lists derived again) and the warm-start features still work."""
    wl = batched["wl"]
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        B.set_tuning(ctx, B.TUNE_DEFER_INSTANCES, 1)
        B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
        B.compute_transition_rates(ctx, 0.0, 0.0, wl.sigma_eV, wl.cutoff_sigmas, instances=INSTANCES)
        B.solve_coupled_bte(ctx, "dragged", wl.tol)
        for i, (_, _, _, ref) in enumerate(standalone):
            c = B.transport_coefficients(ctx, i)
            for key in TENSORS:
                np.testing.assert_array_equal(c[key], batched["coeffs"][i][key])
                assert rel_fro(c[key], ref.coeffs[key]) <= COEFF_RTOL, (i, key)
        again = B.solve_coupled_bte(ctx, "dragged", wl.tol)
        assert again["converged"] == 1
        np.testing.assert_array_equal(B.transport_coefficients(ctx, 1)["sigma"], batched["coeffs"][1]["sigma"])
        import torch
        f = torch.empty((B.num_states(ctx), B.NFEAT), dtype=torch.float32, device="cuda")
        B.state_features(ctx, 2, f.data_ptr())
        torch.cuda.synchronize()
        assert torch.isfinite(f).all()
