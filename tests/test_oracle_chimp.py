"""Pins of the oracle's electron-charged-impurity (e-chimp) channel, Eqs. |g^e-chimp_q|^2, q_TF^2
and X^e-chimp of "Electrons, phonons, and interactions", and its entry into W^RTA (Matthiessen's
rule): the Thomas-Fermi wave vector against the density of states of the closed-form band, the
symmetry of the elastic kernel, point-group invariance (wedge = full zone), the exact n Z^2
scaling, a brute-force golden-rule loop written from the closed-form band, and the RTA rate sum.
CPU only."""
import dataclasses

import numpy as np

import oracle as O
from paper_2109_08547_gb300 import synthetic as S

IMP = S.Impurities(n_cm3=(1.0e19,), Z=(1.0,), eps_r=11.7)


def _sc1(n=8, nsym_full=True, T_K=300.0, imp=IMP):
    return dataclasses.replace(S.workload_sc1(n=n, nsym_full=nsym_full, T_K=T_K), chimp=imp)


def _states(P):
    """The BTE's electron states: (irreducible window k, active band)."""
    return np.array([(k, b) for k in O.ibz_window_points(P) for b in range(P.eps.shape[1]) if P.active[k, b]],
                    dtype=np.int64).reshape(-1, 2)


def _cosine_band(frac):
    """The one-band model's closed form, eps = -2 t sum_a cos(2 pi k_a), t = 1 eV."""
    return -2.0 * np.cos(2.0 * np.pi * frac).sum(axis=-1)


def test_thomas_fermi_wave_vector_is_the_density_of_states_at_mu():
    """Degenerate limit of Eq. q_TF^2: q_TF^2 = e^2 d_s D(mu) / (eps0 eps V) with D the density of
    states per cell and spin, here from a 160^3 histogram of the closed-form band (the window of
    +-0.05 eV around mu = 0.3 eV, where the cosine band's density is smooth).  The oracle sums
    f(1 - f) over a 48^3 mesh at 600 K (kT = 52 meV; on a 24^3 mesh the clustered energies of the
    regular grid still leave the sum 19 % low)."""
    wl = _sc1(n=48, T_K=600.0)
    P = O.prepare(wl)
    q2 = O.thomas_fermi_q2(P, IMP)
    g = (np.arange(160) + 0.5) / 160.0
    fr = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    e = _cosine_band(fr)
    mu, half = wl.mu_eV, 0.05
    D_per_eV = np.count_nonzero(np.abs(e - mu) < half) / (e.size * 2 * half)   # per cell and spin
    V = 27.0 * O.ANGSTROM ** 3
    expect = wl.model.spin_deg * O.E_CHARGE ** 2 * (D_per_eV / O.E_CHARGE) / (O.EPS0 * IMP.eps_r * V)
    assert abs(q2 / expect - 1.0) < 0.02, (q2, expect)


def _full_zone_kernel(n=7):
    """K between all active states of the one-band model without point symmetry, with the
    final states in the order of the initial ones."""
    wl = _sc1(n=n, nsym_full=False)
    P = O.prepare(wl)
    states = np.argwhere(P.active)
    K, fk, fb = O.chimp_kernel(P, states)
    assert np.array_equal(np.stack([fk, fb], 1), states)
    return P, states, K


def test_elastic_kernel_is_symmetric():
    """X^e-chimp / f(1-f) from a to b equals that from b to a: |g_q|^2 depends on |q| and
    [k - k'] = -[k' - k], the transport factor and the Gaussian are symmetric (an odd mesh, no
    point on the zone boundary where the centred k is ambiguous)."""
    _, _, K = _full_zone_kernel()
    assert np.max(np.abs(K - K.T)) <= 1e-12 * np.max(np.abs(K))
    assert np.count_nonzero(K) > 0
    # forward scattering is suppressed: a state does not scatter into itself
    assert np.all(np.diag(K) == 0.0)


def test_chimp_rates_are_point_group_invariant_and_wedge_equals_full_zone():
    """W^chimp(S k) = W^chimp(k) for the 48 operations of O_h (the full-zone model on a 7^3
    mesh), and the irreducible path of the symmetric model gives the same rates at its
    representatives."""
    P, states, K = _full_zone_kernel()
    W = K.sum(axis=1)
    n = np.array(P.wl.kmesh)
    Wk = {int(k): w for (k, _), w in zip(states, W)}
    for Sop in P.wl.model.sym_rot:
        for k, w in list(Wk.items()):
            ki = np.mod(P.kidx[k] @ Sop.T, n)
            k2 = int(O.flat_index(ki[None], tuple(n))[0])
            assert abs(Wk[k2] - w) <= 1e-12 * abs(w)
    wl_s = _sc1(n=7, nsym_full=True)
    Ps = O.prepare(wl_s)
    sts = _states(Ps)
    Ws = O.chimp_rates(Ps, sts)
    for (k, _), w in zip(sts, Ws):
        assert abs(Wk[int(k)] - w) <= 1e-12 * abs(w)


def test_rates_scale_as_concentration_times_charge_squared():
    """The carriers set q_TF, the dopants only the prefactor: W is linear in n_i and quadratic
    in Z_i, and two species add."""
    P1 = O.prepare(_sc1())
    st = _states(P1)
    W1 = O.chimp_rates(P1, st)
    for imp, factor in ((S.Impurities((3.0e19,), (1.0,), 11.7), 3.0), (S.Impurities((1.0e19,), (2.0,), 11.7), 4.0),
                        (S.Impurities((1.0e19, 2.0e19), (1.0, 1.0), 11.7), 3.0)):
        P2 = O.prepare(_sc1(imp=imp))
        np.testing.assert_allclose(O.chimp_rates(P2, st), factor * W1, rtol=1e-12)


def test_rates_equal_a_golden_rule_loop_from_the_closed_form_band():
    """Brute force on a 6^3 mesh from the closed-form band, written out per pair: for every
    irreducible window state, the sum over all k' of 2 pi/(hbar N_k) |g|^2 (1 - cos) delta."""
    wl = _sc1(n=6)
    P = O.prepare(wl)
    st = _states(P)
    W = O.chimp_rates(P, st)
    n = 6
    a = 3.0e-10
    fr = np.array([[i, j, k] for i in range(n) for j in range(n) for k in range(n)], dtype=float) / n
    e = _cosine_band(fr)
    f = 1.0 / (np.exp((e - wl.mu_eV) / (O.KB_EVK * wl.T_K)) + 1.0)
    beta = 1.0 / (O.KB_EVK * O.E_CHARGE * wl.T_K)
    qtf2 = 2.0 * O.E_CHARGE ** 2 * beta * np.sum(f * (1 - f)) / (n ** 3 * a ** 3 * O.EPS0 * 11.7)
    lo, hi = wl.window
    for (k, _), w in zip(st, W):
        total = 0.0
        fk = fr[k] - np.floor(fr[k] + 0.5)
        kv = 2 * np.pi / a * fk
        for kp in range(n ** 3):
            if not (lo <= e[kp] <= hi):
                continue
            fq = fr[kp] - fr[k]
            fq = fq - np.floor(fq + 0.5)
            q2 = np.sum((2 * np.pi / a * fq) ** 2)
            U = O.E_CHARGE / (O.EPS0 * 11.7 * (q2 + qtf2))
            g2 = 1e25 * U ** 2 / a ** 3
            fkp = fr[kp] - np.floor(fr[kp] + 0.5)
            kpv = 2 * np.pi / a * fkp
            den = np.linalg.norm(kv) * np.linalg.norm(kpv)
            tf = 1.0 - (kv @ kpv / den if den > 0 else 0.0)
            x = e[kp] - e[k]
            s = wl.sigma_eV
            d = np.exp(-x * x / (2 * s * s)) / (s * np.sqrt(2 * np.pi)) if abs(x) <= 8 * s else 0.0
            total += 2 * np.pi / (O.HBAR_EVS * n ** 3) * g2 * tf * d
        assert abs(total - w) <= 1e-12 * max(abs(w), 1e-300), (k, total, w)


def test_rta_rates_obey_matthiessens_rule_and_conductivity_drops():
    """Eq. W^RTA: the e-chimp rate adds to the e-ph one state by state; the extra out-scattering
    (not offset by in-scattering, which the transport factor already stands for) lowers sigma."""
    wl = _sc1()
    P = O.prepare(wl)
    R = O.transition_rates(P)
    with_imp = O.solve_coupled_bte(P, R, level="dragged")
    P0 = dataclasses.replace(P, wl=dataclasses.replace(wl, chimp=None))
    without = O.solve_coupled_bte(P0, R, level="dragged")
    Wc = O.chimp_rates(P, with_imp.states)
    np.testing.assert_allclose(with_imp.W_e - without.W_e, Wc, rtol=1e-12)
    assert with_imp.coeffs["sigma"][0, 0] < without.coeffs["sigma"][0, 0]
