"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Bands/phonons to 1e-12 eV, integer tables bit-exact, rates per entry to 1e-10 relative
(floor 1e-6 of the largest rate), RTA rates to 1e-10, coefficient tensors to 1e-8
(relative Frobenius).  Cases span the symmetric IBZ path, the brute-force full BZ, the
4-band/6-branch model, a non-cubic mesh, a k mesh finer than the q mesh, the full-size
24^3 model on sampled rows, an empty window and call-order errors."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2109_08547_gb300 import binding as B
from paper_2109_08547_gb300 import synthetic as S
from _parity import COEFF_RTOL, compare_rates, gpu_rate_table, oracle_rate_table, rel_fro

pytestmark = pytest.mark.gpu

TENSORS = ("sigma", "sigmaS", "S", "alpha_el", "kappa0_el", "kappa_el", "alpha_ph", "kappa_ph")


def _cases():
    cs = S.workload_cscl4(6)
    return {
        "sc1-oh": S.workload_sc1(),
        "sc1-full": S.workload_sc1(nsym_full=False),
        "cscl4-6": cs,
        "cscl4-ragged": dataclasses.replace(cs, name="cscl4-6x4x5", kmesh=(6, 4, 5), qmesh=(6, 4, 5)),
        "cscl4-ratio2": dataclasses.replace(cs, name="cscl4-k8-q4", kmesh=(8, 8, 8), qmesh=(4, 4, 4)),
        # eight bands under O_h, on equal meshes and with the k mesh twice the q mesh
        "sc8-oh": S.workload_sc8(6),
        "sc8-k8-q4": S.workload_sc8(8, ratio=2),
    }


CASES = _cases()


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    wl = CASES[request.param]
    P = O.prepare(wl)
    # no state may sit within rounding of a window edge (the two sides would disagree on it)
    assert np.min(np.abs(P.eps[..., None] - np.array(wl.window))) > 1e-9
    R = O.transition_rates(P)
    ctx = B.Context(0)
    B.set_wannier_model(ctx, wl.model)
    mesh = B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
    rates = B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas)
    yield dict(name=request.param, wl=wl, P=P, R=R, ctx=ctx, mesh=mesh, rates=rates)
    ctx.close()


def test_bands_and_phonons(case):
    P, ctx = case["P"], case["ctx"]
    np.testing.assert_allclose(B.get_array(ctx, "eps").reshape(P.eps.shape), P.eps, rtol=0, atol=1e-12)
    v = B.get_array(ctx, "vel").reshape(P.vel.shape)
    np.testing.assert_allclose(v, P.vel, rtol=0, atol=1e-9 * np.abs(P.vel).max())
    np.testing.assert_allclose(B.get_array(ctx, "omega").reshape(P.w.shape), P.w, rtol=0, atol=1e-12)
    vp = B.get_array(ctx, "vph").reshape(P.vph.shape)
    np.testing.assert_allclose(vp, P.vph, rtol=0, atol=1e-9 * np.abs(P.vph).max())


def test_window_ibz_and_pairs(case):
    P, R, ctx, mesh = case["P"], case["R"], case["ctx"], case["mesh"]
    assert mesh["n_active_states"] == int(P.active.sum())
    np.testing.assert_array_equal(B.get_array(ctx, "ibz_rep"), P.rep)
    np.testing.assert_array_equal(B.get_array(ctx, "ibz_op"), P.op)
    np.testing.assert_array_equal(B.get_array(ctx, "ibzw_list"), R.ibz_win)
    assert mesh["n_pairs"] == R.n_pairs
    assert case["rates"]["n_tuples"] == R.n_tuples
    assert case["rates"]["n_entries"] == len(R.Xp)


def test_transition_rates(case):
    compare_rates(gpu_rate_table(case["ctx"], case["wl"]), oracle_rate_table(case["R"]), case["P"])


# The k 8^3 / q 4^3 case leaves states whose partners are almost only themselves (q = 0
# optical processes inside the delta cut): the plain iteration has spectral radius ~ 1
# there, so both sides are compared after the same fixed number of iterations.
CAPS = {"cscl4-ratio2": dict(max_outer=3, max_inner=40)}


@pytest.mark.parametrize("level", ["rta", "dragless", "partial", "dragged"])
def test_coefficients(case, level):
    wl, P, R, ctx = case["wl"], case["P"], case["R"], case["ctx"]
    caps = CAPS.get(case["name"], {})
    ref = O.solve_coupled_bte(P, R, level=level, **caps)
    info = B.solve_coupled_bte(ctx, level, wl.tol, allow_noconv=bool(caps), **caps)
    got = B.transport_coefficients(ctx)
    assert info["converged"] == int(ref.converged)
    if not caps:
        assert ref.converged
    for key in TENSORS:
        err = rel_fro(got[key], ref.coeffs[key])
        assert err <= COEFF_RTOL, f"{level} {key}: {err:.3e}"
    # RTA rates per state and per mode
    We = B.get_array(ctx, "w_e")
    nb = wl.model.nb
    st = {tuple(s): i for i, s in enumerate(ref.states)}
    ibzw = B.get_array(ctx, "ibzw_list")
    for idx in range(len(We)):
        key = (int(ibzw[idx // nb]), idx % nb)
        if key in st:
            np.testing.assert_allclose(We[idx], ref.W_e[st[key]], rtol=1e-10)
        else:
            assert We[idx] == 0.0
    np.testing.assert_allclose(B.get_array(ctx, "w_ph").reshape(P.w.shape), ref.W_ph, rtol=1e-10,
                               atol=1e-10 * ref.W_ph.max())


def test_repeat_is_bit_identical():
    wl = S.workload_sc1()
    ctx, r1 = _run(wl)
    ctx2, r2 = _run(wl)
    for key in TENSORS:
        np.testing.assert_array_equal(r1.coeffs[key], r2.coeffs[key])
    ctx.close()
    ctx2.close()


def _run(wl, **kw):
    ctx = B.Context(0)
    B.set_wannier_model(ctx, wl.model)
    return ctx, B.run_path(ctx, wl, **kw)


def test_full_size_sampled_rows():
    """The 4-band model on its full 24^3 meshes: every entry of two sampled irreducible rows
    against the oracle, detailed balance on those rows against the reverse rows, and the
    coupled solve converging with the Kelvin-Onsager identity checked on the result."""
    wl = S.workload_cscl4(24)
    ctx = B.Context(0)
    B.set_wannier_model(ctx, wl.model)
    res = B.run_path(ctx, wl, level="dragged")
    assert res.solve["converged"] == 1
    gpu = gpu_rate_table(ctx, wl)
    P = O.prepare(wl)
    ibzw = O.ibz_window_points(P)
    rows = [int(ibzw[len(ibzw) // 3]), int(ibzw[(2 * len(ibzw)) // 3])]
    R = O.transition_rates(P, ks=rows)
    compare_rates(gpu, oracle_rate_table(R), P, rows=set(rows))
    beta = 1.0 / (O.KB_EVK * wl.T_K)
    mq = O.minus_q(P, R.iq)
    n_checked = 0
    for i in range(len(R.Xp)):
        if R.Xp[i] <= 0:
            continue
        rev = gpu.get((int(R.ikp[i]), int(R.n[i]), int(mq[i]), int(R.m[i]), int(R.s[i])))
        assert rev is not None
        x = P.eps[R.ikp[i], R.n[i]] - P.eps[R.ik[i], R.m[i]] - P.w[R.iq[i], R.s[i]]
        np.testing.assert_allclose(R.Xp[i] / rev[1], np.exp(beta * x), rtol=1e-9)
        n_checked += 1
    assert n_checked > 50
    c = res.coeffs
    # sigmaS[I_diff] = alpha_el / T holds for any J; with the correction the remaining gap is
    # the part of alpha_ph/T orthogonal to sigmaS[I_drag]
    assert np.all(np.isfinite(c["sigma"])) and np.linalg.det(c["sigma"]) > 0
    ctx.close()


def test_empty_window():
    wl = dataclasses.replace(S.workload_sc1(), window=(50.0, 60.0))
    ctx = B.Context(0)
    B.set_wannier_model(ctx, wl.model)
    res = B.run_path(ctx, wl, level="dragged")
    assert res.mesh["n_active_states"] == 0 and res.rates["n_entries"] == 0
    for key in ("sigma", "sigmaS", "alpha_el", "kappa0_el"):
        assert np.all(res.coeffs[key] == 0.0)
    ctx.close()


def test_call_order_and_arguments():
    wl = S.workload_sc1()
    ctx = B.Context(0)
    with pytest.raises(B.EphbError) as e:
        B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window)
    assert e.value.status == B.ESTATE
    B.set_wannier_model(ctx, wl.model)
    with pytest.raises(B.EphbError) as e:
        B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV)
    assert e.value.status == B.ESTATE
    with pytest.raises(B.EphbError) as e:
        B.build_meshes_ibz(ctx, (8, 8, 8), (3, 3, 3), wl.window)
    assert e.value.status == B.EINVAL
    with pytest.raises(B.EphbError) as e:
        B.build_meshes_ibz(ctx, (8, 8, 6), (8, 8, 6), wl.window)   # O_h needs a cubic mesh
    assert e.value.status == B.EINVAL
    B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window)
    with pytest.raises(B.EphbError) as e:
        B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, precision=B.SPLIT_TF32)
    assert e.value.status == B.EINVAL
    with pytest.raises(B.EphbError) as e:
        B.solve_coupled_bte(ctx)
    assert e.value.status == B.ESTATE
    B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV)
    info = B.solve_coupled_bte(ctx, "dragged", 1e-14, max_outer=2, max_inner=3, allow_noconv=True)
    assert info["status"] == B.ENOCONV and info["converged"] == 0
    ctx.close()


# ----------------------------------------------------------------- tensor-core contraction
# FP64-grade slicing must meet the FP64 tolerances.  The 3-slice mixed mode is held to the
# mixed-precision target: coefficients within 1e-6 of the FP64 oracle, rates within 1e-6 of
# the largest rate (its per-coefficient error is reported by the benchmark).
MIXED_RTOL = 1e-6


@pytest.mark.parametrize("mode", ["fp64-sliced", "split-bf16"])
def test_tensor_core_contraction(case, mode):
    wl, P, R, ctx = case["wl"], case["P"], case["R"], case["ctx"]
    info = B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas,
                                      precision=B.PRECISIONS[mode])
    assert info["n_entries"] == len(R.Xp)
    assert info["tensor_flops"] > 0
    gpu = gpu_rate_table(ctx, wl)
    ora = oracle_rate_table(R)
    if mode == "fp64-sliced":
        compare_rates(gpu, ora, P)
    else:
        xmax = max(max(abs(v[0]), abs(v[1])) for v in ora.values())
        worst = max(max(abs(gpu[k][0] - v[0]), abs(gpu[k][1] - v[1])) for k, v in ora.items()) / xmax
        assert worst <= MIXED_RTOL, f"mixed-precision rate error {worst:.3e} of the largest rate"
    caps = CAPS.get(case["name"], {})
    ref = O.solve_coupled_bte(P, R, level="dragged", **caps)
    B.solve_coupled_bte(ctx, "dragged", wl.tol, allow_noconv=bool(caps), **caps)
    got = B.transport_coefficients(ctx)
    tol = COEFF_RTOL if mode == "fp64-sliced" else MIXED_RTOL
    for key in TENSORS:
        err = rel_fro(got[key], ref.coeffs[key])
        assert err <= tol, f"{mode} {key}: {err:.3e}"
