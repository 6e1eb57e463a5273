"""Pins of the FP64 oracle against things other than itself: closed forms, finite
differences, unitarity, Hermiticity and symmetry identities, detailed balance, a
brute-force full-BZ run, a dense direct solve of the same linear system, sum rules
and the Kelvin-Onsager identity.  CPU only."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2109_08547_gb300 import synthetic as S

HB = O.HBAR_EVS
A_M = O.ANGSTROM


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ------------------------------------------------------------------ bands and phonons

def test_sc1_bands_closed_form(sc1_prepared):
    """Nearest-neighbour tight binding: eps = -2t sum cos(k_a a), v_a = (2ta/hbar) sin(k_a a)."""
    P = sc1_prepared
    kc = P.kidx / np.array(P.wl.kmesh)
    eps = -2.0 * np.cos(2 * np.pi * kc).sum(axis=1)
    np.testing.assert_allclose(P.eps[:, 0], eps, atol=1e-13)
    v = (2.0 * 3.0 / HB) * np.sin(2 * np.pi * kc) * A_M
    np.testing.assert_allclose(P.vel[:, 0, :], v, atol=1e-9 * np.abs(v).max())


def test_sc1_phonons_closed_form(sc1_prepared):
    """Nearest-neighbour springs: hbar w_a = w_max |sin(q_a a/2)| with Cartesian eigenvectors;
    v = (w_max a / 2 hbar) cos(q_a a/2) sgn(sin) along a, zero across."""
    P = sc1_prepared
    W, a = 0.030, 3.0
    qc = P.qidx / np.array(P.wl.qmesh)
    w_exact = W * np.abs(np.sin(np.pi * qc))
    np.testing.assert_allclose(P.w, np.sort(w_exact, axis=1), atol=1e-12)
    for q in range(P.Nq):
        order = np.argsort(w_exact[q], kind="stable")
        we = w_exact[q, order]
        if np.min(np.diff(we)) < 1e-6 or we[0] < 1e-4:
            continue  # degenerate or Gamma-like: covered by averaging tests
        for s, ax in enumerate(order):
            v = np.zeros(3)
            v[ax] = (W * a / (2 * HB)) * np.cos(np.pi * qc[q, ax]) * np.sign(np.sin(np.pi * qc[q, ax])) * A_M
            np.testing.assert_allclose(P.vph[q, s], v, atol=1e-9 * abs(v[ax]))


def test_multiband_velocity_matches_finite_difference():
    """Hellmann-Feynman v = (1/hbar) d eps/dk against a central difference of the eigenvalues
    (electrons) and of hbar w (phonons) of the 4-band / 6-branch model."""
    m = S.model_cscl4()
    rng = np.random.default_rng(7)
    k = rng.random((12, 3))
    h = 1e-5
    e0, _, v = O.electron_bands(m, k, 1e-6)
    w0, _, vp = O.phonon_modes(m, k, 1e-6, 1e-4)
    a = 3.0
    for d in range(3):
        dk = np.zeros(3)
        dk[d] = h
        ep, _, _ = O.electron_bands(m, k + dk, 1e-6)
        em, _, _ = O.electron_bands(m, k - dk, 1e-6)
        wp, _, _ = O.phonon_modes(m, k + dk, 1e-6, 1e-4)
        wm, _, _ = O.phonon_modes(m, k - dk, 1e-6, 1e-4)
        dkc = 2 * np.pi * h / a   # cartesian step (1/Angstrom)
        fd = (ep - em) / (2 * dkc) / HB * A_M
        fdw = (wp - wm) / (2 * dkc) / HB * A_M
        ok = np.min(np.abs(np.diff(e0, axis=1)), axis=1) > 1e-3
        np.testing.assert_allclose(v[ok, :, d], fd[ok], rtol=1e-5, atol=1e-6 * np.abs(v).max())
        okw = np.min(np.abs(np.diff(w0, axis=1)), axis=1) > 1e-4
        np.testing.assert_allclose(vp[okw, :, d], fdw[okw], rtol=1e-5, atol=1e-6 * np.abs(vp).max())


def test_acoustic_sum_rule_and_stability():
    m = S.model_cscl4()
    q = np.vstack([np.zeros((1, 3)), np.random.default_rng(3).random((50, 3))])
    w, _, _ = O.phonon_modes(m, q, 1e-6, 1e-4)
    assert np.all(w[0, :3] < 1e-8) and np.all(w[0, 3:] > 1e-3)
    Dq = np.einsum("qr,rab->qab", np.exp(2j * np.pi * q @ m.Rd.T), m.D_R)
    assert np.min(np.linalg.eigvalsh(Dq)) > -1e-12
    # zone-centre optical frequency set by the model (0.060 eV)
    np.testing.assert_allclose(w[0, 3:], 0.060, rtol=1e-12)


# ------------------------------------------------------------------ Bloch vertex

def _r0_only(m):
    g = np.zeros_like(m.g_R)
    ie = [i for i, r in enumerate(m.Rge) if not r.any()][0]
    ip = [i for i, r in enumerate(m.Rgp) if not r.any()][0]
    g[ie, ip] = m.g_R[ie, ip]
    return dataclasses.replace(m, g_R=g), g[ie, ip]


def test_vertex_unitarity_with_R0_couplings():
    """Only g(0,0) nonzero => G(k,q) = g(0,0) for all k,q, and the band/branch rotations are
    unitary: sum_{m,n,s} (w_s/w_ref) |g|^2 = sum_alpha (m_bar/m_alpha) ||g(0,0)_alpha||_F^2."""
    wl = S.workload_cscl4(4)
    m0, g00 = _r0_only(wl.model)
    wl = dataclasses.replace(wl, model=m0, window=(-100.0, 100.0))
    P = O.prepare(wl)
    mass = np.repeat(m0.mass_amu, 3)
    expect = np.sum(np.abs(g00) ** 2 * (mass.mean() / mass)[None, None, :])
    k = 5
    qs = np.array([1, 7, 22, 41, 63])
    kps = O.kplusq(P, k, qs)
    g2 = O.bloch_vertex_sq(P, k, qs, kps)
    for i, q in enumerate(qs):
        assert np.all(P.w[q] > 1e-4)
        tot = np.sum(g2[i] * (P.w[q] / m0.omega_ref_eV)[None, None, :])
        np.testing.assert_allclose(tot, expect, rtol=1e-12)


def test_vertex_one_band_R0_is_constant(sc1_prepared):
    """One band, Cartesian phonon eigenvectors: |g_s|^2 = (w_ref/w_s) |g(0,0)|^2 exactly."""
    m0, g00 = _r0_only(sc1_prepared.wl.model)
    P = O.prepare(dataclasses.replace(sc1_prepared.wl, model=m0))
    k = 3
    qs = np.arange(P.Nq)
    kps = O.kplusq(P, k, qs)
    g2 = O.bloch_vertex_sq(P, k, qs, kps)
    ok = P.w > 1e-4
    expect = (m0.omega_ref_eV / P.w[ok]) * np.abs(g00[0, 0, 0]) ** 2
    np.testing.assert_allclose(g2[:, 0, 0, :][ok], expect, rtol=1e-12)


@pytest.mark.parametrize("which", ["sc1", "cscl4"])
def test_vertex_hermiticity(which):
    """|g_mn(k,q)| = |g_nm(k+q,-q)| (absorption and emission share the vertex)."""
    wl = S.workload_sc1() if which == "sc1" else S.workload_cscl4(4)
    P = O.prepare(wl)
    rng = np.random.default_rng(11)
    for k in rng.integers(0, P.Nk, 4):
        qs = rng.integers(0, P.Nq, 6)
        kps = O.kplusq(P, k, qs)
        g2 = O.bloch_vertex_sq(P, k, qs, kps)
        mqs = O.minus_q(P, qs)
        for i in range(len(qs)):
            back = O.bloch_vertex_sq(P, kps[i], mqs[i:i + 1], np.array([k]))[0]
            ok = P.w[qs[i]] > 1e-4
            np.testing.assert_allclose(g2[i][:, :, ok], np.swapaxes(back, 0, 1)[:, :, ok],
                                       rtol=1e-9, atol=1e-12 * g2.max())


def test_vertex_cubic_symmetry(sc1_prepared):
    """|g(Sk, Sq)|^2 = |g(k,q)|^2 for every O_h operation of the symmetric one-band model."""
    P = sc1_prepared
    nk = np.array(P.wl.kmesh)
    rng = np.random.default_rng(5)
    for k in rng.integers(0, P.Nk, 3):
        qs = rng.integers(0, P.Nq, 5)
        g2 = O.bloch_vertex_sq(P, k, qs, O.kplusq(P, k, qs))
        for Sop in P.wl.model.sym_rot[::7]:
            kS = O.flat_index(np.mod(Sop @ P.kidx[k], nk), P.wl.kmesh)
            qS = O.flat_index(np.mod(P.qidx[qs] @ Sop.T, nk), P.wl.qmesh)
            g2S = O.bloch_vertex_sq(P, kS, qS, O.kplusq(P, kS, qS))
            np.testing.assert_allclose(g2S, g2, rtol=1e-10, atol=1e-14 * g2.max())


def test_degenerate_average_is_gauge_invariant(sc1_prepared):
    """Rotating phonon eigenvectors by a random unitary inside a degenerate subspace leaves
    the subspace-averaged |g|^2 unchanged (q on the body diagonal: triply degenerate)."""
    P = sc1_prepared
    q = O.flat_index(np.array([1, 1, 1]), P.wl.qmesh)
    k = 0
    g_ref = O.bloch_vertex_sq(P, k, np.array([q]), O.kplusq(P, k, np.array([q])))
    rng = np.random.default_rng(2)
    Z = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    Q, _ = np.linalg.qr(Z)
    u2 = P.u.copy()
    u2[q] = u2[q] @ Q
    P2 = dataclasses.replace(P, u=u2)
    g_rot = O.bloch_vertex_sq(P2, k, np.array([q]), O.kplusq(P2, k, np.array([q])))
    np.testing.assert_allclose(g_rot, g_ref, rtol=1e-12)


# ------------------------------------------------------------------ rates

def test_sc1_counts(sc1_prepared, sc1_rates):
    """Window/IBZ/cut bookkeeping of the one-band 8^3 case: 92 active FBZ states, 4 IBZ
    points with an active band, 368 (k,q) pairs, 574 entries within the 8-sigma cut
    (1148 when X+ and X- are counted separately)."""
    assert sc1_prepared.active.sum() == 92
    assert len(sc1_rates.ibz_win) == 4
    assert sc1_rates.n_pairs == 368
    assert len(sc1_rates.Xp) == 574


def test_detailed_balance(sc1_full_prepared, sc1_full_rates):
    """X+(mk -> nk' | q) / X-(nk' -> mk | -q) = exp(beta (eps_nk' - eps_mk - hbar w_sq))."""
    P, R = sc1_full_prepared, sc1_full_rates
    key = {(a, b, c, d, e): i for i, (a, b, c, d, e) in enumerate(zip(R.ik, R.m, R.iq, R.n, R.s))}
    beta = 1.0 / (O.KB_EVK * P.wl.T_K)
    checked = 0
    mq = O.minus_q(P, R.iq)
    for i in range(len(R.Xp)):
        if R.Xp[i] <= 0:
            continue
        j = key.get((R.ikp[i], R.n[i], mq[i], R.m[i], R.s[i]))
        assert j is not None
        x = P.eps[R.ikp[i], R.n[i]] - P.eps[R.ik[i], R.m[i]] - P.w[R.iq[i], R.s[i]]
        np.testing.assert_allclose(R.Xp[i] / R.Xm[j], np.exp(beta * x), rtol=1e-10)
        checked += 1
    assert checked > 100


def test_rates_vanish_beyond_cut(sc1_rates, sc1_prepared):
    P, R = sc1_prepared, sc1_rates
    xp = P.eps[R.ikp, R.n] - P.eps[R.ik, R.m] - P.w[R.iq, R.s]
    xm = xp + 2 * P.w[R.iq, R.s]
    cut = P.wl.cutoff_sigmas * P.wl.sigma_eV
    assert np.all(R.Xp[np.abs(xp) > cut] == 0) and np.all(R.Xm[np.abs(xm) > cut] == 0)
    assert np.all((np.abs(xp) <= cut) | (np.abs(xm) <= cut))


# ------------------------------------------------------------------ BTE and coefficients

@pytest.mark.parametrize("level", ["rta", "dragless", "dragged"])
def test_ibz_path_equals_full_bz(sc1_prepared, sc1_rates, sc1_full_prepared, sc1_full_rates, level):
    """IBZ representatives + symmetry rotations + phonon fold reproduce the brute-force
    full-BZ calculation (no symmetry) for RTA, dragless and dragged solutions."""
    a = O.solve_coupled_bte(sc1_prepared, sc1_rates, level=level)
    b = O.solve_coupled_bte(sc1_full_prepared, sc1_full_rates, level=level)
    assert a.converged and b.converged
    for key in ("sigma", "sigmaS", "alpha_el", "kappa0_el", "alpha_ph", "kappa_ph"):
        np.testing.assert_allclose(a.coeffs[key], b.coeffs[key], rtol=1e-8,
                                   atol=1e-8 * np.abs(b.coeffs[key]).max() + 1e-300)
    # electron RTA rates agree state by state
    full = {tuple(s): w for s, w in zip(b.states, b.W_e)}
    for (k, m), w in zip(a.states, a.W_e):
        np.testing.assert_allclose(w, full[(k, m)], rtol=1e-11)
    np.testing.assert_allclose(a.W_ph, b.W_ph, rtol=1e-11)


def test_cubic_tensors_are_isotropic(sc1_prepared, sc1_rates):
    r = O.solve_coupled_bte(sc1_prepared, sc1_rates, level="dragged")
    for key in ("sigma", "sigmaS", "kappa_el", "kappa_ph", "alpha_ph"):
        t = r.coeffs[key]
        d = np.diag(t)
        np.testing.assert_allclose(d, d[0], rtol=1e-12)
        assert np.max(np.abs(t - np.diag(d))) < 1e-12 * abs(d[0])
    assert r.coeffs["S"][0, 0] < 0, "electron-like carriers above mid-band give S < 0"


def test_rta_is_first_iterate(sc1_prepared, sc1_rates):
    """Iteration 0 is the RTA: I = (eps-mu)/T v/W, J = v/W, F = (hbar w/T) v/W, G = 0."""
    P = sc1_prepared
    r = O.solve_coupled_bte(P, sc1_rates, level="rta")
    ks, bs = r.states[:, 0], r.states[:, 1]
    v = P.vel[ks, bs]
    np.testing.assert_allclose(r.J, v / r.W_e[:, None], rtol=1e-15)
    np.testing.assert_allclose(r.I, ((P.eps[ks, bs] - P.wl.mu_eV) / P.wl.T_K)[:, None] * v / r.W_e[:, None],
                               rtol=1e-15)
    ok = P.w > P.wl.omega_min_eV
    np.testing.assert_allclose(r.F[ok], (P.w[ok] / P.wl.T_K)[:, None] * P.vph[ok] / r.W_ph[ok][:, None], rtol=1e-15)
    assert np.all(r.G == 0)
    d = O.solve_coupled_bte(P, sc1_rates, level="dragged")
    for key in r.coeffs:
        np.testing.assert_array_equal(d.rta_coeffs[key], r.coeffs[key])


def test_kelvin_onsager_identity_after_correction(sc1_prepared, sc1_rates):
    """After the correction sigma S = (alpha_el + alpha_ph)/T holds (isotropic case), and
    sigmaS[I_diff] = alpha_el/T is an identity for I_diff = (eps-mu) J/(eT)."""
    P = sc1_prepared
    r = O.solve_coupled_bte(P, sc1_rates, level="dragged", ko=True)
    c = r.coeffs
    T = P.wl.T_K
    np.testing.assert_allclose(c["sigmaS"], (c["alpha_el"] + c["alpha_ph"]) / T, rtol=1e-11,
                               atol=1e-11 * np.abs(c["sigmaS"]).max())
    sp = O.StateSpace(P, sc1_rates)
    I_diff = ((sp.eps - P.wl.mu_eV) / T)[:, None] * r.J
    np.testing.assert_allclose(sp.electron_tensors(I_diff, r.J)["sigmaS"], c["alpha_el"] / T, rtol=1e-13,
                               atol=1e-13 * np.abs(c["alpha_el"]).max() / T)
    assert 0.0 < r.lambdas[-1] < 2.0


def test_sigma_f_sum_rule():
    """Units and BZ weights of sigma: with a constant relaxation time tau (J = v tau) the
    mesh sum sum_k f(1-f)/kT v_x^2 equals sum_k f d2eps/dk_x^2 / hbar^2 (integration by
    parts over the periodic zone), so sigma_xx = d_s e tau 2 t a^2 <f cos(k_x a)> / (V hbar^2)
    (t, hbar in eV units).  Hot, wide-window case on the O_h IBZ so that the symmetrisation
    of the sums is pinned too."""
    wl = S.workload_sc1(n=40)
    wl = dataclasses.replace(wl, T_K=20000.0, mu_eV=-2.0, window=(-6.5, 6.5))
    P = O.prepare(wl)
    sp = O.StateSpace(P)
    tau = 1e-14
    J = sp.v * tau
    I = ((sp.eps - wl.mu_eV) / wl.T_K)[:, None] * J
    sig = sp.electron_tensors(I, J)["sigma"]
    kc = P.kidx / np.array(wl.kmesh)
    f = O.fermi(P.eps[:, 0], wl.mu_eV, wl.T_K)
    a_m = 3.0 * A_M
    V = (3.0 * A_M) ** 3
    expect = 2.0 * O.E_CHARGE * tau * 2.0 * 1.0 * a_m ** 2 * np.mean(f * np.cos(2 * np.pi * kc[:, 0])) / (V * HB ** 2)
    np.testing.assert_allclose(np.diag(sig), expect, rtol=1e-7)


def test_kappa_ph_classical_limit():
    """Units of kappa_ph: constant tau, k_B T >> hbar w, so (hbar w)^2 n(1+n) -> (k_B T)^2 and
    kappa_xx = (k_B tau / V) (1/N) sum_qs v_x^2.  For the nearest-neighbour spring model the
    x-polarised branch carries v_x = (w_max a/2 hbar) cos(q_x a/2); when it is degenerate with
    d-1 other branches the subspace-averaged velocities give that branch's v_x^2 / d in
    total.  Modes with w = 0 are excluded."""
    n = 8
    wl = dataclasses.replace(S.workload_sc1(n=n), T_K=3.0e5)
    P = O.prepare(wl)
    sp = O.StateSpace(P)
    tau = 1e-12
    F = (P.w / wl.T_K)[..., None] * P.vph * tau
    kap = sp.phonon_tensors(F, np.zeros_like(F))["kappa_ph"]
    kB = O.KB_EVK * O.E_CHARGE
    vmax = 0.030 * 3.0 / (2 * HB) * A_M
    qc = P.qidx / n
    wa = 0.030 * np.abs(np.sin(np.pi * qc))
    tot = 0.0
    for q in range(P.Nq):
        if wa[q, 0] <= 1e-4:
            continue
        d = np.count_nonzero(np.abs(wa[q] - wa[q, 0]) < 1e-6)
        tot += np.cos(np.pi * qc[q, 0]) ** 2 / d
    expect = kB * tau / (3.0 * A_M) ** 3 * vmax ** 2 * tot / P.Nq
    np.testing.assert_allclose(np.diag(kap), expect, rtol=1e-6)


def test_fixed_point_equals_dense_solve(sc1_full_prepared, sc1_full_rates):
    """With the Kelvin-Onsager step off, the converged coupled iteration solves the linear
    system of the four BTEs.  Assemble that system as a dense matrix from the rate list
    and solve it directly (least squares: electron-number conservation makes it singular
    along constant I), then compare the coefficients."""
    P, R = sc1_full_prepared, sc1_full_rates
    it = O.solve_coupled_bte(P, R, level="dragged", ko=False, tol=1e-12)
    assert it.converged
    sp = O.StateSpace(P, R)
    ne, nq, nbr = len(sp.states), P.Nq, sp.nbr
    nph = nq * nbr
    ds = P.wl.model.spin_deg
    W_e, W_ph = it.W_e, it.W_ph
    ok = P.w.ravel() > P.wl.omega_min_eV
    M = np.zeros((ne + nph, ne + nph))
    for e in range(len(R.Xp)):
        i, j = sp.row[e], sp.col[e]
        qs = R.iq[e] * nbr + R.s[e]
        mqs = sp.mq[e] * nbr + R.s[e]
        c = 1.0 / (sp.ff[i] * W_e[i])
        M[i, j] += c * (R.Xp[e] + R.Xm[e])
        M[i, ne + qs] -= c * R.Xp[e]
        M[i, ne + mqs] += c * R.Xm[e]
        y = R.Xp[e] * P.Nq / P.Nk
        cp = ds / (sp.nn1.ravel()[qs] * W_ph.ravel()[qs])
        M[ne + qs, j] += cp * y
        M[ne + qs, i] -= cp * y
    A = np.eye(ne + nph) - M
    keep = np.concatenate([np.ones(ne, bool), ok])
    A = A[np.ix_(keep, keep)]
    T, mu = P.wl.T_K, P.wl.mu_eV
    I0 = ((sp.eps - mu) / T)[:, None] * sp.v / W_e[:, None]
    J0 = sp.v / W_e[:, None]
    F0 = ((P.w / T)[..., None] * P.vph / np.where(W_ph > 0, W_ph, 1.0)[..., None]).reshape(nph, 3)
    bT = np.vstack([I0, F0[ok]])
    bE = np.vstack([J0, np.zeros((ok.sum(), 3))])
    xT = np.linalg.lstsq(A, bT, rcond=None)[0]
    xE = np.linalg.lstsq(A, bE, rcond=None)[0]
    F = np.zeros((nph, 3))
    G = np.zeros((nph, 3))
    F[ok] = xT[ne:]
    G[ok] = xE[ne:]
    c = O.coefficients_from_responses(sp, xT[:ne], xE[:ne], F.reshape(nq, nbr, 3), G.reshape(nq, nbr, 3))
    for key in ("sigma", "sigmaS", "alpha_el", "kappa0_el", "alpha_ph", "kappa_ph"):
        np.testing.assert_allclose(it.coeffs[key], c[key], rtol=1e-7, atol=1e-7 * np.abs(c[key]).max())


def test_eight_band_model_symmetry_ibz_equals_full_bz():
    """The 8-band O_h model: the irreducible-wedge solution with the 48 operations equals the
    full-zone solution without them (which needs the model's O_h invariance of H and the
    covariance of g), on a 4^3 mesh at the dragged level."""
    import oracle as O
    from paper_2109_08547_gb300 import synthetic as SY
    res = []
    for full in (True, False):
        wl = SY.workload_sc8(4, nsym_full=full)
        P = O.prepare(wl)
        R = O.transition_rates(P)
        res.append(O.solve_coupled_bte(P, R, level="dragged"))
    assert res[0].converged and res[1].converged
    for key in ("sigma", "sigmaS", "alpha_el", "kappa0_el", "alpha_ph", "kappa_ph"):
        a, b = res[0].coeffs[key], res[1].coeffs[key]
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b), key


# ------------------------------------------------------------------ absolute rate scale and mesh ratio

def _sc1_r0_workload(n_k, n_q, sym=True, **kw):
    """The one-band cubic model with only the R = 0 coupling kept: every |g_s|^2 is then
    (w_ref / w_s) |g(0,0)|^2, so the rates follow from closed-form bands and phonons."""
    wl = S.workload_sc1(n_k, nsym_full=sym)
    m0, g00 = _r0_only(wl.model)
    return dataclasses.replace(wl, model=m0, qmesh=(n_q,) * 3, **kw), abs(g00[0, 0, 0]) ** 2


def _sc1_closed(wl):
    """Closed-form eps(k) (nearest-neighbour band, t = 1 eV) and the three Cartesian phonon
    branches w_a(q) = w_max |sin(pi q_a / n_q)| of the one-band model."""
    nk, nq = np.array(wl.kmesh), np.array(wl.qmesh)
    eps = lambda ki: -2.0 * np.cos(2 * np.pi * ki / nk).sum(axis=-1)
    wq = lambda qi: 0.030 * np.abs(np.sin(np.pi * qi / nq))
    return eps, wq


@pytest.mark.parametrize("n_k,n_q", [(8, 8), (8, 4)])
def test_rate_sums_equal_golden_rule_brute_force(n_k, n_q):
    """Absolute scale of Eq. X^e-ph on equal and ratio-2 meshes.  With a constant |g|^2 the
    summed absorption / emission rates of an initial state are golden-rule sums over the
    final states k' = k + q, q running over the N_q points of the phonon mesh:
      sum X^{+/-}(k) = (2 pi / hbar) (1/N_q) sum_{q, a} |g_a|^2 f_k (1 - f_k') {n, 1+n} delta(x),
    with delta the unit-normalised Gaussian of standard deviation sigma (zero beyond the cut).
    The loop below uses the closed-form band and phonon energies, visits every q of the
    phonon mesh directly (no irreducible wedge, no pair tables) and checks every irreducible
    state to 1e-12.  A wrong 2 pi, hbar, 1/N normalisation or Gaussian normalisation fails."""
    wl, g2 = _sc1_r0_workload(n_k, n_q)
    P = O.prepare(wl)
    R = O.transition_rates(P)
    eps, wq = _sc1_closed(wl)
    T, mu, sig, cut = wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas * wl.sigma_eV
    kT = O.KB_EVK * T
    lo, hi = wl.window
    qall = O.mesh_indices(wl.qmesh)
    r = n_k // n_q
    gauss = lambda x: np.where(np.abs(x) <= cut, np.exp(-x * x / (2 * sig * sig)) / (sig * np.sqrt(2 * np.pi)), 0.0)
    checked = 0
    for k in R.ibz_win:
        ki = P.kidx[k]
        e = eps(ki)
        kpi = ki[None, :] + r * qall
        ep = eps(kpi)
        act = (ep >= lo) & (ep <= hi)
        f, fp = 1 / (np.exp((e - mu) / kT) + 1), 1 / (np.exp((ep - mu) / kT) + 1)
        sp = sm = 0.0
        for a in range(3):
            w = wq(qall)[:, a]
            ok = act & (w > wl.omega_min_eV)
            n = 1.0 / np.expm1(w[ok] / kT)
            base = (2 * np.pi / HB) / qall.shape[0] * g2 * (wl.model.omega_ref_eV / w[ok]) * f * (1 - fp[ok])
            sp += np.sum(base * n * gauss(ep[ok] - e - w[ok]))
            sm += np.sum(base * (1 + n) * gauss(ep[ok] - e + w[ok]))
        sel = R.ik == k
        np.testing.assert_allclose(R.Xp[sel].sum(), sp, rtol=1e-12)
        np.testing.assert_allclose(R.Xm[sel].sum(), sm, rtol=1e-12)
        checked += 1
    assert checked == len(R.ibz_win) > 0


@pytest.mark.parametrize("n_k,n_q", [(8, 8), (8, 4)])
def test_phonon_rta_rate_equals_brute_force_over_all_k(n_k, n_q):
    """Eq. W^RTA of the phonons on equal and ratio-2 meshes: the electron part of a mode's
    rate is d_s sum_{k in FBZ} Y / (n(1+n)) with Y = (2 pi / hbar)(1/N_k) |g|^2 f_k (1 - f_k+q) n
    delta: a golden-rule sum over every k of the electron mesh, each weighted 1/N_k.  The loop
    below visits all N_k points (the oracle builds the same sum from irreducible rows and the
    symmetry fold) with closed-form energies, and adds the background rate."""
    wl, g2 = _sc1_r0_workload(n_k, n_q)
    P = O.prepare(wl)
    R = O.transition_rates(P)
    res = O.solve_coupled_bte(P, R, level="rta")
    eps, wq = _sc1_closed(wl)
    T, mu, sig, cut = wl.T_K, wl.mu_eV, wl.sigma_eV, wl.cutoff_sigmas * wl.sigma_eV
    kT = O.KB_EVK * T
    lo, hi = wl.window
    m = wl.model
    kall = P.kidx
    e = eps(kall)
    f = 1 / (np.exp((e - mu) / kT) + 1)
    act = (e >= lo) & (e <= hi)
    r = n_k // n_q
    for q in range(P.Nq):
        qi = P.qidx[q]
        w_all = wq(qi)
        order = np.argsort(w_all, kind="stable")
        ep = eps(kall + r * qi[None, :])
        fp = 1 / (np.exp((ep - mu) / kT) + 1)
        both = act & (ep >= lo) & (ep <= hi)
        for s, a in enumerate(order):
            w = w_all[a]
            if w <= wl.omega_min_eV:
                continue
            n = 1.0 / np.expm1(w / kT)
            x = ep[both] - e[both] - w
            d = np.where(np.abs(x) <= cut, np.exp(-x * x / (2 * sig * sig)) / (sig * np.sqrt(2 * np.pi)), 0.0)
            Y = (2 * np.pi / HB) / P.Nk * g2 * (m.omega_ref_eV / w) * f[both] * (1 - fp[both]) * n * d
            expect = m.spin_deg * Y.sum() / (n * (1 + n)) + m.bg_rate_coeff * (w / m.bg_omega_ref_eV) ** 2 * (T / m.bg_T_ref)
            np.testing.assert_allclose(res.W_ph[q, s], expect, rtol=1e-12)


def test_rta_rates_do_not_depend_on_the_mesh_ratio():
    """[A3] from the physics side: the RTA rates are Brillouin-zone integrals, so an 8^3 k mesh
    with a 4^3 or an 8^3 phonon mesh must give the same rates up to discretisation error.
    Normalising X by 1/N_k instead of 1/N_q, or Y by 1/N_q instead of 1/N_k, would change one
    of them by a factor 8.  Mean electron rate over the active states and the n(1+n)-weighted
    zone average of the phonon rates' electron part, wide Gaussian (50 meV) so the mesh sums
    are smooth."""
    out = []
    for n_q in (8, 4):
        wl, _ = _sc1_r0_workload(8, n_q, sigma_eV=0.05)
        P = O.prepare(wl)
        res = O.solve_coupled_bte(P, O.transition_rates(P), level="rta")
        m = wl.model
        bg = m.bg_rate_coeff * (P.w / m.bg_omega_ref_eV) ** 2 * (wl.T_K / m.bg_T_ref)
        nb = O.bose(P.w, wl.T_K)
        ok = P.w > wl.omega_min_eV
        out.append((res.W_e.mean(), np.sum(((res.W_ph - bg) * nb * (1 + nb))[ok]) / P.Nq))
    (we8, wp8), (we4, wp4) = out
    assert 0.8 < we4 / we8 < 1.25
    assert 0.6 < wp4 / wp8 < 1.6


def test_gaussian_delta_is_unit_normalised_with_sigma_as_standard_deviation():
    """[A10] delta(x) integrates to 1 inside the 8-sigma cut (up to the erfc(8/sqrt 2) ~ 1e-15
    tail), its second moment is sigma^2, its peak 1/(sigma sqrt(2 pi)), and it is exactly zero
    beyond the cut."""
    sig, cut = 0.010, 8.0
    x = np.linspace(-cut * sig, cut * sig, 400001)
    d = O.gaussian_delta(x, sig, cut)
    h = x[1] - x[0]
    trap = lambda y: h * (y.sum() - 0.5 * (y[0] + y[-1]))
    np.testing.assert_allclose(trap(d), 1.0, rtol=1e-10)
    np.testing.assert_allclose(trap(d * x * x), sig * sig, rtol=1e-9)
    np.testing.assert_allclose(O.gaussian_delta(np.array([0.0]), sig, cut)[0], 1.0 / (sig * np.sqrt(2 * np.pi)), rtol=1e-15)
    assert O.gaussian_delta(np.array([cut * sig * (1 + 1e-12)]), sig, cut)[0] == 0.0


def test_kelvin_onsager_identity_on_ratio_two_mesh():
    """The Kelvin-Onsager identities after the correction on an 8^3 k / 4^3 q mesh (O_h
    wedge).  The plain iteration barely contracts on this small ratio-2 mesh, so a fixed
    number of iterations is run: the identity holds after every correction step."""
    wl = dataclasses.replace(S.workload_sc1(8), qmesh=(4, 4, 4))
    P = O.prepare(wl)
    R = O.transition_rates(P)
    r = O.solve_coupled_bte(P, R, level="dragged", ko=True, max_outer=3, max_inner=40)
    c = r.coeffs
    T = wl.T_K
    np.testing.assert_allclose(c["sigmaS"], (c["alpha_el"] + c["alpha_ph"]) / T, rtol=1e-11,
                               atol=1e-11 * np.abs(c["sigmaS"]).max())
    sp = O.StateSpace(P, R)
    I_diff = ((sp.eps - wl.mu_eV) / T)[:, None] * r.J
    np.testing.assert_allclose(sp.electron_tensors(I_diff, r.J)["sigmaS"], c["alpha_el"] / T, rtol=1e-13,
                               atol=1e-13 * np.abs(c["alpha_el"]).max() / T)


def _dense_coupled_operator(P, R, W_e, W_ph):
    """The linear map of one sweep of the coupled BTEs (KO step off), assembled entry by entry
    from the rate list: electron rows (self and drag terms of Eqs. dI^S, dI^D) and phonon rows
    (Eq. dF^D, each X^+ entry seen from the phonon with Y = X^+ N_q / N_k)."""
    sp = O.StateSpace(P, R)
    ne, nbr = len(sp.states), sp.nbr
    nph = P.Nq * nbr
    ds = P.wl.model.spin_deg
    M = np.zeros((ne + nph, ne + nph))
    for e in range(len(R.Xp)):
        i, j = sp.row[e], sp.col[e]
        qs = R.iq[e] * nbr + R.s[e]
        mqs = sp.mq[e] * nbr + R.s[e]
        c = 1.0 / (sp.ff[i] * W_e[i])
        M[i, j] += c * (R.Xp[e] + R.Xm[e])
        M[i, ne + qs] -= c * R.Xp[e]
        M[i, ne + mqs] += c * R.Xm[e]
        y = R.Xp[e] * P.Nq / P.Nk
        cp = ds / (sp.nn1.ravel()[qs] * W_ph.ravel()[qs])
        M[ne + qs, j] += cp * y
        M[ne + qs, i] -= cp * y
    return sp, M, ne, nph


def test_partial_level_is_one_drag_update_then_exact_electrons(sc1_full_prepared, sc1_full_rates):
    """The partially decoupled iterate ("Coupled and decoupled BTEs", iterate 1): the phonons
    take one drag update from the RTA electrons, F = F0 + dF^D[I0], G = dG^D[J0], and the
    electron equations are then solved exactly against those fixed phonons (KO step off).
    Reference: the dense operator applied once to the RTA, then a direct least-squares solve
    of the electron block."""
    P, R = sc1_full_prepared, sc1_full_rates
    it = O.solve_coupled_bte(P, R, level="partial", ko=False, tol=1e-12)
    assert it.converged and it.outer_iters == 1
    sp, M, ne, nph = _dense_coupled_operator(P, R, it.W_e, it.W_ph)
    ok = P.w.ravel() > P.wl.omega_min_eV
    T, mu = P.wl.T_K, P.wl.mu_eV
    I0 = ((sp.eps - mu) / T)[:, None] * sp.v / it.W_e[:, None]
    J0 = sp.v / it.W_e[:, None]
    F0 = ((P.w / T)[..., None] * P.vph / np.where(it.W_ph > 0, it.W_ph, 1.0)[..., None]).reshape(nph, 3)
    F0[~ok] = 0.0
    F1 = F0 + M[ne:, :ne] @ I0
    G1 = M[ne:, :ne] @ J0
    F1[~ok] = 0.0
    G1[~ok] = 0.0
    A = np.eye(ne) - M[:ne, :ne]
    I = np.linalg.lstsq(A, I0 + M[:ne, ne:] @ F1, rcond=None)[0]
    J = np.linalg.lstsq(A, J0 + M[:ne, ne:] @ G1, rcond=None)[0]
    c = O.coefficients_from_responses(sp, I, J, F1.reshape(P.Nq, sp.nbr, 3), G1.reshape(P.Nq, sp.nbr, 3))
    for key in ("sigma", "sigmaS", "alpha_el", "kappa0_el", "alpha_ph", "kappa_ph"):
        np.testing.assert_allclose(it.coeffs[key], c[key], rtol=1e-7, atol=1e-7 * np.abs(c[key]).max())
    # and the partial iterate differs from both the RTA and the converged dragged answer
    d = O.solve_coupled_bte(P, R, level="dragged", ko=False, tol=1e-12)
    assert np.linalg.norm(it.coeffs["sigma"] - it.rta_coeffs["sigma"]) > 1e-6 * np.linalg.norm(it.coeffs["sigma"])
    assert np.linalg.norm(it.coeffs["kappa_ph"] - d.coeffs["kappa_ph"]) > 1e-9 * np.linalg.norm(d.coeffs["kappa_ph"])


# ------------------------------------------------------------------ the 8-band fine-mesh drag model

def test_cscl8_band_edges_on_the_80_mesh():
    """The 8-band semiconductor's gap is 1.0 eV on the 80^3 mesh: the oracle's bands on every
    irreducible point give the closed-form VBM (top valence band at Gamma) and CBM (lowest
    conduction band at X) to 1e-12 eV, the conduction minimum sits at the X points, and no
    state lies within 1e-9 eV of a window edge."""
    wl = S.workload_cscl8(80, 40, r_half=1)
    vbm, cbm = S.cscl8_band_edges()
    kidx = O.mesh_indices(wl.kmesh)
    nn = np.array(wl.kmesh)
    images = np.stack([O.flat_index(np.mod(kidx @ Sop.T.astype(np.int64), nn), wl.kmesh) for Sop in wl.model.sym_rot])
    reps = np.unique(images.min(axis=0))
    assert len(reps) == 12341       # C(43, 3): the O_h wedge of an 80^3 mesh
    e, _, _ = O.electron_bands(wl.model, kidx[reps] / nn, wl.degen_tol_eV)
    np.testing.assert_allclose(e[:, :4].max(), vbm, atol=1e-12)
    np.testing.assert_allclose(e[:, 4:].min(), cbm, atol=1e-12)
    np.testing.assert_allclose(e[:, 4:].min() - e[:, :4].max(), 1.0, atol=1e-12)
    kmin = kidx[reps[np.argmin(e[:, 4])]]
    assert sorted(kmin.tolist()) == [0, 0, 40]          # X = (1/2, 0, 0)
    assert np.min(np.abs(e[..., None] - np.array(wl.window))) > 1e-9
    # the window holds conduction states only
    act = (e >= wl.window[0]) & (e <= wl.window[1])
    assert act[:, :4].sum() == 0 and act.sum() > 100


def test_cscl8_couplings_are_oh_covariant_and_hermitian_pair_symmetric():
    """The coupling generator's two symmetry steps, checked entry by entry on a 5^3 grid:
    g^{kappa a}(Re, Rp) = sum_b S_ba g^{kappa b}(S Re, S(Rp + tau_kappa) - tau_kappa) for all 48
    operations (the B atom shifts cell under S), and g_{m'n'}(Re, Rp) = conj g_{n'm'}(-Re, Rp - Re)."""
    m = S.model_cscl8(r_half=2)
    grid = m.Rge
    idx = {tuple(v): i for i, v in enumerate(grid)}
    g = m.g_R.reshape(len(grid), len(grid), 8, 8, 2, 3)
    rng = np.random.default_rng(3)
    tau = np.array([0.5, 0.5, 0.5])
    n_checked = 0
    for Sop in m.sym_rot:
        for _ in range(40):
            a, b, kap = rng.integers(0, len(grid)), rng.integers(0, len(grid)), rng.integers(0, 2)
            re, rp = grid[a], grid[b]
            if kap == 1 and np.any(rp == 2):
                assert np.all(g[a, b, :, :, 1] == 0)
                continue
            rp2 = np.rint(Sop @ (rp + kap * tau) - kap * tau).astype(int)
            rhs = np.einsum("ba,mnb->mna", Sop.astype(float), g[idx[tuple(Sop @ re)], idx[tuple(rp2)], :, :, kap])
            np.testing.assert_allclose(g[a, b, :, :, kap], rhs, atol=1e-17)
            n_checked += 1
    assert n_checked > 1000
    for _ in range(500):
        a, b = rng.integers(0, len(grid)), rng.integers(0, len(grid))
        p = tuple(grid[b] - grid[a])
        if p in idx:
            partner = np.conj(np.swapaxes(g[idx[tuple(-grid[a])], idx[p]], 0, 1))
            for kap in (0, 1):
                if kap == 1 and (np.any(grid[b] == 2) or np.any(np.array(p) == 2)):
                    continue
                np.testing.assert_allclose(g[a, b, :, :, kap], partner[:, :, kap], atol=1e-17)


def test_cscl8_irreducible_wedge_equals_full_zone():
    """The 8-band 2-atom O_h model (small coupling grid): irreducible-wedge rates, RTA,
    dragless and dragged iterates (a fixed number of iterations) equal the full-zone ones
    without symmetry, which needs H(SR) = H(R), the O_h phonons and the covariance of g with
    the B atom's cell shift."""
    m1 = S.model_cscl8(r_half=1)
    res = []
    for full in (True, False):
        wl = S.workload_cscl8(12, 12, model=m1, nsym_full=full)
        P = O.prepare(wl)
        R = O.transition_rates(P)
        res.append([O.solve_coupled_bte(P, R, level=lv, max_outer=4, max_inner=30) for lv in ("rta", "dragless",
                                                                                               "dragged")])
    for a, b in zip(*res):
        for key in ("sigma", "sigmaS", "alpha_el", "kappa0_el", "alpha_ph", "kappa_ph"):
            nb_ = np.linalg.norm(b.coeffs[key])
            if nb_ > 0:
                assert np.linalg.norm(a.coeffs[key] - b.coeffs[key]) <= 1e-11 * nb_, key


def test_cscl8_detailed_balance():
    """Detailed balance of the 8-band 2-atom model (full zone, small coupling grid, window widened
    to 0.9 eV above the CBM): X+(mk -> nk' | q) / X-(nk' -> mk | -q) = exp(beta (eps' - eps - hbar w))
    for every pair of entries above 1e-6 of the largest rate (below that, couplings that the
    symmetry makes vanish leave rounding-level rates whose ratio means nothing)."""
    wl = S.workload_cscl8(8, 8, r_half=1, nsym_full=False, above_cbm_eV=0.9)
    P = O.prepare(wl)
    R = O.transition_rates(P)
    key = {(a, b, c, d, e): i for i, (a, b, c, d, e) in enumerate(zip(R.ik, R.m, R.iq, R.n, R.s))}
    beta = 1.0 / (O.KB_EVK * wl.T_K)
    mq = O.minus_q(P, R.iq)
    floor = 1e-6 * max(R.Xp.max(), R.Xm.max())
    n = 0
    for i in range(len(R.Xp)):
        if R.Xp[i] <= floor:
            continue
        j = key.get((R.ikp[i], R.n[i], mq[i], R.m[i], R.s[i]))
        assert j is not None
        if R.Xm[j] <= floor:
            continue
        x = P.eps[R.ikp[i], R.n[i]] - P.eps[R.ik[i], R.m[i]] - P.w[R.iq[i], R.s[i]]
        np.testing.assert_allclose(R.Xp[i] / R.Xm[j], np.exp(beta * x), rtol=1e-9)
        n += 1
    assert n > 500


# ------------------------------------------------------------------ tetrahedron delta ([A22])

def test_tetra_corner_weights_closed_forms():
    """Corner weights of one linear tetrahedron: their sum is the tetrahedron density of
    states in closed form in each of the three energy ranges (Bloechl's expressions), it
    integrates to 1 over [e_min, e_max], every corner's weight integrates to 1/4 (the mean of its
    barycentric coordinate), and its first moment is (e_c + sum_j e_j) / 20 (the mean of
    lambda_c e over the tetrahedron)."""
    e = np.array([0.3, -0.2, 1.1, 0.5])
    es = np.sort(e)
    e21, e31, e41 = es[1] - es[0], es[2] - es[0], es[3] - es[0]
    e32, e42, e43 = es[2] - es[1], es[3] - es[1], es[3] - es[2]
    for E in (-0.1, 0.05, 0.2):
        np.testing.assert_allclose(O.tetra_corner_weights(e, E).sum(), 3 * (E - es[0]) ** 2 / (e21 * e31 * e41),
                                   rtol=1e-13)
    for E in (0.31, 0.4, 0.49):
        D = (3 * e21 + 6 * (E - es[1]) - 3 * (e31 + e42) * (E - es[1]) ** 2 / (e32 * e42)) / (e31 * e41)
        np.testing.assert_allclose(O.tetra_corner_weights(e, E).sum(), D, rtol=1e-13)
    for E in (0.6, 0.9, 1.05):
        np.testing.assert_allclose(O.tetra_corner_weights(e, E).sum(), 3 * (es[3] - E) ** 2 / (e41 * e42 * e43),
                                   rtol=1e-13)
    Es = np.linspace(es[0], es[3], 200001)
    W = np.array([O.tetra_corner_weights(e, E) for E in Es])
    h = Es[1] - Es[0]
    trap = lambda y: h * (y.sum(axis=0) - 0.5 * (y[0] + y[-1]))
    np.testing.assert_allclose(trap(W).sum(), 1.0, rtol=1e-8)
    np.testing.assert_allclose(trap(W), 0.25, rtol=1e-7)
    np.testing.assert_allclose(trap(W * Es[:, None]), (e + e.sum()) / 20.0, rtol=1e-7, atol=1e-9)
    assert np.all(O.tetra_corner_weights(e, es[0] - 1e-9) == 0) and np.all(O.tetra_corner_weights(e, es[3]) == 0)


def test_tetra_point_weights_give_the_density_of_states():
    """sum_q w(q) over a 12^3 mesh of eps(q) - E, eps the nearest-neighbour band, is the zone
    average of delta(E - eps): the density of states per cell, here against a histogram of the
    band on a 240^3 half-shifted mesh (bins of +-0.05 eV) within 3 % (the linear tetrahedron
    error on the coarse mesh; a wrong normalisation would be off by a factor 4, 6 or N).  The
    weights are invariant under the cubic operations (four-diagonal average)."""
    n = 12
    idx = O.mesh_indices((n, n, n))
    eps = -2.0 * np.cos(2 * np.pi * idx / n).sum(axis=1)
    nf = 240
    c = np.cos(2 * np.pi * (np.arange(nf) + 0.5) / nf)
    ef = -2.0 * (c[:, None, None] + c[None, :, None] + c[None, None, :])
    ops = S.oh_group()
    for E in (-3.1, 0.83):
        w = O.tetra_point_weights(eps - E, (n, n, n), np.arange(n ** 3))
        ref = np.count_nonzero(np.abs(ef - E) < 0.05) / (nf ** 3 * 0.1)
        np.testing.assert_allclose(w.sum(), ref, rtol=0.03)
        for Sop in ops[::5]:
            img = O.flat_index(np.mod(idx @ Sop.T, n), (n, n, n))
            np.testing.assert_allclose(w[img], w, rtol=1e-12, atol=1e-15 * w.max())


def test_tetra_rates_ibz_path_equals_full_bz():
    """Tetrahedron delta on the one-band cubic model: the irreducible-wedge rates and RTA and
    dragged coefficients equal the full-zone ones (the four-diagonal weights are cubic
    invariant)."""
    res = []
    for full in (True, False):
        wl = dataclasses.replace(S.workload_sc1(8, nsym_full=full), delta="tetra")
        P = O.prepare(wl)
        R = O.transition_rates(P)
        res.append([O.solve_coupled_bte(P, R, level=lv) for lv in ("rta", "dragged")])
    for a, b in zip(*res):
        assert a.converged and b.converged
        for key in ("sigma", "sigmaS", "alpha_el", "kappa0_el", "alpha_ph", "kappa_ph"):
            assert np.linalg.norm(a.coeffs[key] - b.coeffs[key]) <= 1e-9 * np.linalg.norm(b.coeffs[key]), key


@pytest.mark.parametrize("n_k,n_q", [(8, 8), (8, 4)])
def test_tetra_rate_sums_equal_brute_force(n_k, n_q):
    """Rates with the tetrahedron delta on equal and ratio-2 meshes: with the constant coupling
    of the one-band model (R = 0 only) every irreducible state's summed X+ and X- equal a direct
    loop over all q of the phonon mesh and the three energy-sorted closed-form branches of
    (2 pi / hbar) |g_s|^2 f_k (1 - f_k+q) {n, 1+n} w(q), w the tetrahedron weight of q for
    eps(k + r q') - eps(k) -/+ w_s(q') built from the closed-form band and frequencies (zero below
    omega_min) -- neither the oracle's bands nor its pair tables.  A wrong 2 pi / hbar, N_q or
    weight normalisation, or a weight for the wrong point, fails."""
    wl, g2 = _sc1_r0_workload(n_k, n_q)
    wl = dataclasses.replace(wl, delta="tetra")
    P = O.prepare(wl)
    R = O.transition_rates(P)
    eps, wq = _sc1_closed(wl)
    T, mu = wl.T_K, wl.mu_eV
    kT = O.KB_EVK * T
    lo, hi = wl.window
    qall = O.mesh_indices(wl.qmesh)
    r = n_k // n_q
    wsorted = np.sort(wq(qall), axis=1)
    wz = np.where(wsorted > wl.omega_min_eV, wsorted, 0.0)
    for k in R.ibz_win:
        ki = P.kidx[k]
        e = eps(ki)
        ep = eps(ki[None, :] + r * qall)
        act = (ep >= lo) & (ep <= hi)
        f, fp = 1 / (np.exp((e - mu) / kT) + 1), 1 / (np.exp((ep - mu) / kT) + 1)
        sp = sm = 0.0
        for s in range(3):
            wp = O.tetra_point_weights(ep - e - wz[:, s], wl.qmesh, np.arange(len(qall)))
            wm = O.tetra_point_weights(ep - e + wz[:, s], wl.qmesh, np.arange(len(qall)))
            ok = act & (wsorted[:, s] > wl.omega_min_eV)
            w = wsorted[ok, s]
            n = 1.0 / np.expm1(w / kT)
            base = (2 * np.pi / HB) * g2 * (wl.model.omega_ref_eV / w) * f * (1 - fp[ok])
            sp += np.sum(base * n * wp[ok])
            sm += np.sum(base * (1 + n) * wm[ok])
        sel = R.ik == k
        np.testing.assert_allclose(R.Xp[sel].sum(), sp, rtol=1e-10)
        np.testing.assert_allclose(R.Xm[sel].sum(), sm, rtol=1e-10)
