"""The coupled iteration as one CUDA graph launch with device-driven loops (solve option
device_loop): the same kernels in the same order per instance as the host-driven loop, so the
coefficients, sweep counts and iteration counts must be bit-identical to it, for one instance
and for several (T, mu, window) instances in one launch; and the oracle's coefficients within
the FP64 tolerance ("Coupled and decoupled BTEs", "Transport coefficients")."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2109_08547_gb300 import binding as B
from paper_2109_08547_gb300 import synthetic as SY
from _parity import COEFF_RTOL, rel_fro

pytestmark = pytest.mark.gpu

TENSORS = ("sigma", "sigmaS", "alpha_el", "kappa0_el", "alpha_ph", "kappa_ph")
COUNTS = ("outer_iters", "inner_iters_total", "n_sweeps", "n_sweeps32", "outer_iters32", "converged",
          "n_zero_rate_states")
INSTANCES = [(300.0, 0.0, -0.3, 0.3), (180.0, 0.12, -0.18, 0.42), (460.0, -0.15, -0.45, 0.05),
             (250.0, 0.05, -0.25, 0.35)]


def _solve_both(ctx, level, tol, solve_precision, n_inst=1):
    host = B.solve_coupled_bte(ctx, level, tol, solve_precision=solve_precision)
    hc = [B.transport_coefficients(ctx, i) for i in range(n_inst)]
    dev = B.solve_coupled_bte(ctx, level, tol, solve_precision=solve_precision, device_loop=True)
    dc = [B.transport_coefficients(ctx, i) for i in range(n_inst)]
    return host, hc, dev, dc


def _assert_identical(host, hc, dev, dc):
    for key in COUNTS:
        assert dev[key] == host[key], (key, dev[key], host[key])
    assert dev["residual"] == host["residual"] and dev["lambda"] == host["lambda"]
    for h, d in zip(hc, dc):
        for key in h:
            np.testing.assert_array_equal(d[key], h[key], err_msg=key)


@pytest.mark.parametrize("solve_precision", ["mixed", "fp64"])
@pytest.mark.parametrize("level", ["dragged", "partial", "dragless"])
@pytest.mark.parametrize("name", ["sc1", "cscl4-6"])
def test_device_loop_is_bit_identical_to_host_loop(name, level, solve_precision):
    wl = SY.workload_sc1() if name == "sc1" else SY.workload_cscl4(n=6)
    prec = B.PRECISIONS["fp64-sliced"] if name != "sc1" else B.FP64
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
        B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas, prec)
        host, hc, dev, dc = _solve_both(ctx, level, wl.tol, solve_precision)
        assert host["graph_launches"] == 0 and dev["graph_launches"] == 1
        _assert_identical(host, hc, dev, dc)
        # nothing changed: the same graph is launched again, with the same answer
        again = B.solve_coupled_bte(ctx, level, wl.tol, solve_precision=solve_precision, device_loop=True)
        assert again["graph_reused"] == 1
        np.testing.assert_array_equal(B.transport_coefficients(ctx)["sigma"], dc[0]["sigma"])


def test_device_loop_matches_oracle_on_the_fine_mesh_model():
    """The bench's mode (FP64-grade tensor-core vertex, mixed iteration, device-driven loops)
    on the 8-band / 6-branch drag model at 12^3 k / 6^3 q (widened window) against the oracle."""
    wl = SY.workload_cscl8(12, 6, above_cbm_eV=0.63)
    P = O.prepare(wl)
    R = O.transition_rates(P)
    ref = O.solve_coupled_bte(P, R, level="dragged", ko=True)
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        r = B.run_path(ctx, wl, level="dragged", precision=B.PRECISIONS["fp64-sliced"], solve_precision="mixed",
                       device_loop=True)
    assert r.solve["converged"] == 1 and r.solve["graph_launches"] == 1
    for key in TENSORS:
        assert rel_fro(r.coeffs[key], ref.coeffs[key]) <= COEFF_RTOL, key


@pytest.mark.parametrize("defer", [0, 1])
@pytest.mark.parametrize("solve_precision", ["mixed", "fp64"])
def test_instances_in_one_launch(solve_precision, defer):
    """Four instances with uneven windows: one graph launch solves all of them (one per instance
    when their lists are derived at solve time), bit-identical to the host loop's instance-by-
    instance solves."""
    wl = dataclasses.replace(SY.workload_cscl4(n=6), window=(-0.45, 0.45))
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        if defer:
            B.set_tuning(ctx, B.TUNE_DEFER_INSTANCES, 1)
        B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
        B.compute_transition_rates(ctx, 0.0, 0.0, wl.sigma_eV, wl.cutoff_sigmas, B.PRECISIONS["fp64-sliced"],
                                   instances=INSTANCES)
        host, hc, dev, dc = _solve_both(ctx, "dragged", wl.tol, solve_precision, n_inst=len(INSTANCES))
        assert dev["graph_launches"] == (len(INSTANCES) if defer else 1)
        _assert_identical(host, hc, dev, dc)
        for i in range(len(INSTANCES)):
            h = B.instance_solve_info(ctx, i)
            assert h["converged"] == 1 and h["graph_launches"] == 1


def test_warm_start_in_the_device_loop():
    """A learned start (here: each state's own converged coordinates) applied in the graph's
    prologue gives the host loop's warm-started solve exactly."""
    import torch
    wl = SY.workload_cscl4(n=6)
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
        B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas)
        B.solve_coupled_bte(ctx, "dragged", wl.tol, solve_precision="mixed")
        a = torch.empty((B.num_states(ctx), 2), dtype=torch.float32, device="cuda")
        B.state_targets(ctx, 0, a.data_ptr())
        torch.cuda.synchronize()
        B.set_warm_start(ctx, 0, a.data_ptr())
        host = B.solve_coupled_bte(ctx, "dragged", wl.tol, solve_precision="mixed", warm_start=True)
        hc = B.transport_coefficients(ctx)
        dev = B.solve_coupled_bte(ctx, "dragged", wl.tol, solve_precision="mixed", warm_start=True,
                                  device_loop=True)
        dc = B.transport_coefficients(ctx)
        _assert_identical(host, [hc], dev, [dc])


def test_device_loop_arguments():
    wl = SY.workload_sc1()
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window)
        B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV)
        with pytest.raises(B.EphbError):
            B.solve_coupled_bte(ctx, "dragged", 1e-10, accel=3, device_loop=True)
        with pytest.raises(B.EphbError):
            B.solve_coupled_bte(ctx, "rta", 1e-10, device_loop=True)
        r = B.solve_coupled_bte(ctx, "dragged", 1e-10, device_loop=True)
        assert r["converged"] == 1


@pytest.mark.parametrize("solve_precision", ["mixed", "fp64"])
def test_device_loop_on_an_empty_window(solve_precision):
    """No state in the window: the graph still builds and runs (every conditional body holds a
    kernel) and gives the host loop's zero electron tensors."""
    wl = dataclasses.replace(SY.workload_sc1(), window=(50.0, 60.0))
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
        B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas)
        host, hc, dev, dc = _solve_both(ctx, "dragged", wl.tol, solve_precision)
        assert dev["graph_launches"] == 1
        _assert_identical(host, hc, dev, dc)
        for key in ("sigma", "sigmaS", "alpha_el", "kappa0_el"):
            assert np.all(dc[0][key] == 0.0)
