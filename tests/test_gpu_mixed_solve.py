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
    assert mixed.solve["n_sweeps"] < plain.solve["n_sweeps"], (mixed.solve["n_sweeps"], plain.solve["n_sweeps"])
    for key in TENSORS:
        assert rel_fro(mixed.coeffs[key], ref.coeffs[key]) <= COEFF_RTOL, key


def test_bad_solve_precision():
    wl = SY.workload_sc1()
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window)
        B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV)
        o = B.SolveOptsC(3, 1e-10, 0.0, 10, 10, 1, 0, 7)
        info = B.SolveInfoC()
        assert B.load().ephb_solve_coupled_bte(ctx.handle, B.C.byref(o), B.C.byref(info)) == B.EINVAL
