"""The mixed-precision electron loop (FP64 residual sweeps + FP32 correction sweeps) reaches the
same converged coefficients as the oracle's plain FP64 iteration, with fewer FP64 sweeps."""
import pytest

import oracle as O
from paper_2109_08547_gb300 import binding as B
from paper_2109_08547_gb300 import synthetic as SY
from _parity import COEFF_RTOL, rel_fro

pytestmark = pytest.mark.gpu

TENSORS = ("sigma", "sigmaS", "alpha_el", "kappa0_el", "alpha_ph", "kappa_ph")


@pytest.mark.parametrize("name", ["sc1", "cscl4-6"])
@pytest.mark.parametrize("level", ["dragless", "dragged"])
def test_mixed_solve_matches_oracle(name, level):
    wl = SY.workload_sc1() if name == "sc1" else SY.workload_cscl4(n=6)
    P = O.prepare(wl)
    R = O.transition_rates(P)
    ref = O.solve_coupled_bte(P, R, level=level)
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        plain = B.run_path(ctx, wl, level=level)
        mixed = B.run_path(ctx, wl, level=level, solve_precision="mixed")
    assert mixed.solve["converged"] == 1 and ref.converged
    assert mixed.solve["n_sweeps32"] > 0
    # dragged: the early outer iterations take FP32 phonon-side terms, the last one FP64
    if level == "dragged":
        assert 0 < mixed.solve["outer_iters32"] < mixed.solve["outer_iters"]
    else:
        assert mixed.solve["outer_iters32"] == 0
    assert mixed.solve["n_sweeps"] < plain.solve["n_sweeps"], (mixed.solve["n_sweeps"], plain.solve["n_sweeps"])
    for key in TENSORS:
        assert rel_fro(mixed.coeffs[key], ref.coeffs[key]) <= COEFF_RTOL, key


def test_loose_tolerance_ends_on_fp64_outer_iteration():
    """A tolerance above the FP32 phonon-side switch point: the solve still ends only after an
    outer iteration whose phonon scatter and drag term ran in FP64."""
    import dataclasses
    wl = dataclasses.replace(SY.workload_cscl4(n=6), tol=1e-4)
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        plain = B.run_path(ctx, wl, level="dragged")
        mixed = B.run_path(ctx, wl, level="dragged", solve_precision="mixed")
    assert mixed.solve["converged"] == 1 and plain.solve["converged"] == 1
    assert mixed.solve["outer_iters32"] < mixed.solve["outer_iters"]
    for key in TENSORS:
        assert rel_fro(mixed.coeffs[key], plain.coeffs[key]) <= 1e-3, key


def test_bad_solve_precision():
    wl = SY.workload_sc1()
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window)
        B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV)
        o = B.SolveOptsC(3, 1e-10, 0.0, 10, 10, 1, 0, 7)
        info = B.SolveInfoC()
        assert B.load().ephb_solve_coupled_bte(ctx.handle, B.C.byref(o), B.C.byref(info)) == B.EINVAL


@pytest.mark.parametrize("solve_precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["sc1", "cscl4-6"])
def test_anderson_outer_iteration_matches_oracle(name, solve_precision):
    """Anderson acceleration of the outer iteration: the oracle's (plain iteration's) converged
    coefficients; in fewer outer iterations where the plain iteration contracts slowly (the
    4-band model, residual ratio ~0.7 per outer iteration).  The 1-band model's outer iteration
    contracts ~100x per step, so there is nothing to gain and only correctness is checked."""
    wl = SY.workload_sc1() if name == "sc1" else SY.workload_cscl4(n=6)
    P = O.prepare(wl)
    R = O.transition_rates(P)
    ref = O.solve_coupled_bte(P, R, level="dragged")
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        acc = B.run_path(ctx, wl, level="dragged", solve_precision=solve_precision, accel=3)
    assert acc.solve["converged"] == 1 and ref.converged
    if name != "sc1":
        assert acc.solve["outer_iters"] < 0.5 * ref.outer_iters, (acc.solve["outer_iters"], ref.outer_iters)
    for key in TENSORS:
        assert rel_fro(acc.coeffs[key], ref.coeffs[key]) <= COEFF_RTOL, key


def test_bad_accel_depth():
    wl = SY.workload_sc1()
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window)
        B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV)
        for depth in (-1, B.MAX_ACCEL_DEPTH + 1):
            with pytest.raises(B.EphbError):
                B.solve_coupled_bte(ctx, "dragged", 1e-10, accel=depth)
