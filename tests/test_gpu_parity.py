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


_CSCL8 = []


def _cscl8_model():
    if not _CSCL8:
        _CSCL8.append(S.model_cscl8())
    return _CSCL8[0]


def _cases():
    """name -> workload factory (the 8-band model takes half a minute to build, so nothing is
    built at collection)."""
    cs = lambda: S.workload_cscl4(6)
    return {
        "sc1-oh": lambda: S.workload_sc1(),
        "sc1-full": lambda: S.workload_sc1(nsym_full=False),
        "cscl4-6": cs,
        "cscl4-ragged": lambda: dataclasses.replace(cs(), name="cscl4-6x4x5", kmesh=(6, 4, 5), qmesh=(6, 4, 5)),
        "cscl4-ratio2": lambda: dataclasses.replace(cs(), name="cscl4-k8-q4", kmesh=(8, 8, 8), qmesh=(4, 4, 4)),
        # eight bands under O_h, on equal meshes and with the k mesh twice the q mesh
        "sc8-oh": lambda: S.workload_sc8(6),
        "sc8-k8-q4": lambda: S.workload_sc8(8, ratio=2),
        # the fine-mesh drag model (8 bands, 2 atoms, 7^3 x 7^3 couplings: contraction length
        # 686, the 8-slice tensor-core form) on small meshes with a widened window
        "cscl8-8": lambda: S.workload_cscl8(8, 8, model=_cscl8_model(), above_cbm_eV=0.9),
        "cscl8-k12-q6": lambda: S.workload_cscl8(12, 6, model=_cscl8_model(), above_cbm_eV=0.63),
    }


CASES = _cases()


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    wl = CASES[request.param]()
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
    # frequencies to 1e-12 eV; at the zone centre the acoustic eigenvalues are rounding noise
    # (~1e-18 eV^2, so hbar w ~1e-9 eV or a clipped 0): there both sides only need to be
    # below omega_min, the modes every sum leaves out
    w = B.get_array(ctx, "omega").reshape(P.w.shape)
    keep = P.w > case["wl"].omega_min_eV
    np.testing.assert_allclose(w[keep], P.w[keep], rtol=0, atol=1e-12)
    assert np.all(w[~keep] < 1e-6) and np.all(P.w[~keep] < 1e-6)
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


def test_full_size_cscl8_sampled_rows():
    """The fine-mesh drag model at its full size (80^3 k under O_h, 40^3 q, 7^3 x 7^3 couplings)
    with the benchmark's default flags (FP64-grade 8-slice tensor-core vertex, mixed-precision
    iteration, Anderson depth 3): the irreducible window list against the oracle's, every entry
    of two sampled irreducible rows against the oracle at the FP64 tolerance, detailed balance
    against the reverse entries, and the converged coefficients against the plain FP64 path
    (FP64 vertex, plain FP64 iteration) at 1e-8; the mixed-precision vertex's rates on the same
    rows within 1e-6 of the largest rate and its coefficients within 1e-6."""
    wl = S.workload_cscl8(80, 40, model=_cscl8_model())
    ibzw = O.ibz_window_rows(wl)
    rows = [int(ibzw[len(ibzw) // 3]), int(ibzw[(2 * len(ibzw)) // 3])]
    P = O.prepare_rows(wl, rows)
    R = O.transition_rates(P, ks=rows)
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        fast = B.run_path(ctx, wl, level="dragged", precision=B.FP64_SLICED, solve_precision="mixed", accel=3)
        assert fast.solve["converged"] == 1
        np.testing.assert_array_equal(B.get_array(ctx, "ibzw_list"), ibzw)
        gpu = gpu_rate_table(ctx, wl)
        compare_rates(gpu, oracle_rate_table(R), P, rows=set(rows))
        beta = 1.0 / (O.KB_EVK * wl.T_K)
        mq = O.minus_q(P, R.iq)
        n_checked = 0
        # couplings that the symmetry makes vanish leave rates at the rounding level (~1e-20 of
        # the largest): their ratios carry no information, so only rates above the parity floor
        floor = 1e-6 * max(R.Xp.max(), R.Xm.max())
        for i in range(len(R.Xp)):
            if R.Xp[i] <= floor:
                continue
            rev = gpu.get((int(R.ikp[i]), int(R.n[i]), int(mq[i]), int(R.m[i]), int(R.s[i])))
            if rev is None or rev[1] <= floor:   # k' is not a representative, or a rounding-level rate
                continue
            x = P.eps[R.ikp[i], R.n[i]] - P.eps[R.ik[i], R.m[i]] - P.w[R.iq[i], R.s[i]]
            np.testing.assert_allclose(R.Xp[i] / rev[1], np.exp(beta * x), rtol=1e-9)
            n_checked += 1
        assert n_checked > 20
        plain = B.run_path(ctx, wl, level="dragged", precision=B.FP64, solve_precision="fp64", accel=0)
        assert plain.solve["converged"] == 1
        for key in TENSORS:
            assert rel_fro(fast.coeffs[key], plain.coeffs[key]) <= COEFF_RTOL, key
        mixed = B.run_path(ctx, wl, level="dragged", precision=B.SPLIT_BF16, solve_precision="mixed", accel=3)
        assert mixed.solve["converged"] == 1
        gm = gpu_rate_table(ctx, wl)
        ora = oracle_rate_table(R)
        xmax = max(max(abs(v[0]), abs(v[1])) for v in ora.values())
        worst = max(max(abs(gm[k][0] - v[0]), abs(gm[k][1] - v[1])) for k, v in ora.items()) / xmax
        assert worst <= MIXED_RTOL, worst
        for key in TENSORS:
            assert rel_fro(mixed.coeffs[key], plain.coeffs[key]) <= MIXED_RTOL, key


@pytest.mark.parametrize("name", ["cscl4-6", "sc8-k8-q4", "cscl8-8", "cscl8-k12-q6"])
def test_default_fast_path_matches_oracle(name):
    """The benchmark's default flags end to end (FP64-grade tensor-core vertex, mixed-precision
    iteration, Anderson depth 3 on the outer iteration, tol 1e-10) against the oracle's plain
    iteration: every rate entry at 1e-10 and every coefficient at 1e-8."""
    wl = CASES[name]()
    P = O.prepare(wl)
    R = O.transition_rates(P)
    ref = O.solve_coupled_bte(P, R, level="dragged")
    assert ref.converged
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        r = B.run_path(ctx, wl, level="dragged", precision=B.FP64_SLICED, solve_precision="mixed", accel=3)
        assert r.solve["converged"] == 1
        compare_rates(gpu_rate_table(ctx, wl), oracle_rate_table(R), P)
    for key in TENSORS:
        assert rel_fro(r.coeffs[key], ref.coeffs[key]) <= COEFF_RTOL, key


def _straddle_workload():
    """Two copies of the one-band orbital, on-site energies 0 and 5e-7 eV (degenerate within the
    1e-6 eV tolerance everywhere), couplings g_sc1 x [[1, 0.3], [0.3, 0.7]] (O_h covariant and
    Hermitian-pair symmetric like g_sc1), and a window whose lower edge sits 2.5e-7 eV above the
    states at eps = 0: there every degenerate pair is cut by the edge, its upper band active and
    its lower band not."""
    m1 = S.model_sc1()
    H = np.zeros((m1.H_R.shape[0], 2, 2), dtype=np.complex128)
    for r in range(m1.H_R.shape[0]):
        H[r] = m1.H_R[r, 0, 0] * np.eye(2)
    r0 = [i for i, v in enumerate(m1.Re) if not v.any()][0]
    H[r0] += np.diag([0.0, 5e-7])
    mix = np.array([[1.0, 0.3], [0.3, 0.7]])
    g = m1.g_R[:, :, 0, 0, :][:, :, None, None, :] * mix[None, None, :, :, None]
    m2 = dataclasses.replace(m1, nb=2, H_R=H, g_R=np.ascontiguousarray(g))
    wl = S.workload_sc1()
    return dataclasses.replace(wl, name="sc1x2-straddle", model=m2, window=(2.5e-7, wl.window[1]))


@pytest.mark.parametrize("mode", ["fp64", "fp64-sliced"])
def test_degenerate_subspace_cut_by_the_window_edge(mode):
    """[A9]: |g|^2 is averaged over the whole degenerate subspace, also where the window edge
    cuts it (the oracle averages over all its bands; the GPU path rotates the inactive partner
    too).  Every rate entry at 1e-10, the coefficients at 1e-8."""
    wl = _straddle_workload()
    P = O.prepare(wl)
    assert np.min(np.abs(P.eps[..., None] - np.array(wl.window))) > 1e-9
    cut = (P.active[:, 1] & ~P.active[:, 0]) & (np.abs(P.eps[:, 1] - P.eps[:, 0]) < wl.degen_tol_eV)
    assert cut.sum() > 0
    R = O.transition_rates(P)
    ref = O.solve_coupled_bte(P, R, level="dragged")
    assert ref.converged
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        r = B.run_path(ctx, wl, level="dragged", precision=B.PRECISIONS[mode])
        assert r.solve["converged"] == 1
        compare_rates(gpu_rate_table(ctx, wl), oracle_rate_table(R), P)
    for key in TENSORS:
        assert rel_fro(r.coeffs[key], ref.coeffs[key]) <= COEFF_RTOL, key


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
    # a lattice vector beyond the 32-bit mesh-index arithmetic is refused
    import dataclasses
    far = wl.model.Re.copy()
    far[0, 0] = 70000
    with pytest.raises(B.EphbError) as e:
        B.set_wannier_model(ctx, dataclasses.replace(wl.model, Re=far))
    assert e.value.status == B.EINVAL
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


# ----------------------------------------------------------------- tetrahedron delta
_TETRA_REF = {}


@pytest.mark.parametrize("name,mode", [("sc1-oh", "fp64"), ("sc1-oh", "fp64-sliced"), ("cscl4-6", "fp64-sliced"),
                                       ("cscl8-k12-q6", "fp64"), ("cscl8-k12-q6", "fp64-sliced")])
def test_tetrahedron_delta_matches_oracle(name, mode):
    """The analytic tetrahedron delta ([A22]) on the symmetric, unsymmetric, ratio-2 and 8-band
    cases: the entry sets bit-exact (an entry exists where a weight is positive), every rate at
    1e-10, the RTA and dragged coefficients at 1e-8 (ratio-2: a fixed number of iterations)."""
    if name not in _TETRA_REF:   # the oracle side once per case
        wl = dataclasses.replace(CASES[name](), delta="tetra")
        P = O.prepare(wl)
        R = O.transition_rates(P)
        _TETRA_REF[name] = (wl, P, R, {lv: O.solve_coupled_bte(P, R, level=lv, **CAPS.get(name, {}))
                                       for lv in ("rta", "dragged")})
    wl, P, R, refs = _TETRA_REF[name]
    caps = CAPS.get(name, {})
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window, wl.degen_tol_eV, wl.omega_min_eV)
        info = B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas,
                                          precision=B.PRECISIONS[mode], delta="tetra")
        assert info["n_tuples"] == R.n_tuples
        gpu = gpu_rate_table(ctx, wl)
        ora = oracle_rate_table(R)
        # a tetrahedron whose level set only grazes a corner gives a weight at the rounding level,
        # which either side may see as zero: entries present on one side only must be such
        xmax = max(max(abs(v[0]), abs(v[1])) for v in ora.values())
        for key in set(gpu) ^ set(ora):
            v = gpu.get(key, ora.get(key))
            assert max(abs(v[0]), abs(v[1])) <= 1e-12 * xmax, key
        common = set(gpu) & set(ora)
        compare_rates({k: gpu[k] for k in common}, {k: ora[k] for k in common}, P)
        for level in ("rta", "dragged"):
            ref = refs[level]
            B.solve_coupled_bte(ctx, level, wl.tol, allow_noconv=bool(caps), **caps)
            got = B.transport_coefficients(ctx)
            for key in TENSORS:
                assert rel_fro(got[key], ref.coeffs[key]) <= COEFF_RTOL, (level, key)
