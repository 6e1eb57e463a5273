"""The tile autotuner of the tensor-core contraction: the first call of a context times the
candidate column-chunk widths and keeps one; the rates do not depend on the width chosen
(every column is summed in the same order), so they are bit-identical for every width."""
import numpy as np
import pytest

from paper_2109_08547_gb300 import binding as B
from paper_2109_08547_gb300 import synthetic as SY

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,widths", [("fp64-sliced", (48, 64, 96)), ("split-bf16", (64, 128, 256))])
def test_tile_width_is_tuned_and_result_invariant(precision, widths):
    wl = SY.workload_cscl4(n=6)
    outs = []
    for width in (0,) + widths:
        with B.Context(0) as ctx:
            B.set_wannier_model(ctx, wl.model)
            B.set_tuning(ctx, B.TUNE_TC_COLS, width)
            B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
            r = B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas,
                                           B.PRECISIONS[precision])
            if width == 0:
                assert r["autotuned"] == 1 and r["tc_cols"] in widths
                r2 = B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas,
                                                B.PRECISIONS[precision])
                assert r2["autotuned"] == 0 and r2["tc_cols"] == r["tc_cols"]
            else:
                assert r["autotuned"] == 0 and r["tc_cols"] == width
            outs.append(B.get_array(ctx, "entry_x"))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_bad_width_is_rejected():
    with B.Context(0) as ctx:
        for bad in (8, 100, 512):
            with pytest.raises(B.EphbError):
                B.set_tuning(ctx, B.TUNE_TC_COLS, bad)


def test_wait_timeout_is_reported_and_the_context_recovers():
    """With the tensor-core MMAs withheld the barriers never complete: every bounded wait gives
    up (2 s), the call returns EPHB_ETIMEOUT, and the same context then computes the same rates
    as a fresh one."""
    wl = SY.workload_cscl4(n=6)
    with B.Context(0) as ctx, B.Context(0) as ref:
        for c in (ctx, ref):
            B.set_wannier_model(c, wl.model)
            B.set_tuning(c, B.TUNE_TC_COLS, 96)
            B.build_meshes_ibz(c, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
        B.set_tuning(ctx, B.TUNE_WITHHOLD_MMA, 1)
        with pytest.raises(B.EphbError) as err:
            B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas, B.FP64_SLICED)
        assert err.value.status == B.ETIMEOUT
        B.set_tuning(ctx, B.TUNE_WITHHOLD_MMA, 0)
        B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas, B.FP64_SLICED)
        B.compute_transition_rates(ref, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas, B.FP64_SLICED)
        assert np.array_equal(B.get_array(ctx, "entry_x"), B.get_array(ref, "entry_x"))


@pytest.mark.parametrize("name", ["cscl4-6", "cscl8-k12-q6"])
def test_stage_a_tensor_memory_form_is_bit_identical(name):
    """Stage A with every product reading its A slice from shared memory (the default) and with
    the A slices copied into tensor memory once per K step: the same products in the same
    order, so the rates are bit-identical (7 slices on the 4-band model, 8 on the 7^3-grid
    model)."""
    wl = SY.workload_cscl4(n=6) if name == "cscl4-6" else SY.workload_cscl8(12, 6)
    outs = []
    for tmem_a in (0, 1):
        with B.Context(0) as ctx:
            B.set_wannier_model(ctx, wl.model)
            B.set_tuning(ctx, B.TUNE_STAGE_A_TMEM_A, tmem_a)
            B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
            B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas, B.FP64_SLICED)
            outs.append((B.get_array(ctx, "entry_x"), B.get_array(ctx, "entry_kpns")))
    assert outs[0][0].size > 0
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][0], outs[1][0])
