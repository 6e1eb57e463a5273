"""Pins of the oracle's phonon-isotope (Tamura) channel, Eq. W^ph-x of "Electrons, phonons, and
interactions", and its entry into W^RTA_sq: a closed form from the one-band model's Cartesian
phonons, point-group invariance on a 2-atom model, linearity in g, and Matthiessen's rule in
the solve.  CPU only."""
import dataclasses

import numpy as np

import oracle as O
from paper_2109_08547_gb300 import synthetic as S

G = 2.0e-4


def _sc1(n=8, g=G):
    return dataclasses.replace(S.workload_sc1(n=n), isotopes=(g,))


def test_closed_form_of_cartesian_phonons():
    """The one-band model's phonons are hbar w_a(q) = w_max |sin(pi q_a)| with Cartesian
    eigenvectors, so |xi_s . xi_s'|^2 is 1 for equal directions and 0 otherwise, and by cubic
    symmetry every direction has the same spectrum: W(sq) = pi E^2 g / (2 hbar N_q)
    sum_q' delta(w_max |sin(pi q'_x)| - E), the final modes above omega_min, whatever the
    degenerate group of sq (its average is over directions with the same sum)."""
    wl = _sc1()
    P = O.prepare(wl)
    W = O.isotope_rates(P, (G,))
    n = wl.qmesh[0]
    qx = P.qidx[:, 0] / n
    Ex = 0.030 * np.abs(np.sin(np.pi * qx))
    ok_final = Ex > wl.omega_min_eV
    for q in range(P.Nq):
        for s in range(3):
            E = P.w[q, s]
            if not E > wl.omega_min_eV:
                assert W[q, s] == 0.0
                continue
            d = O.gaussian_delta(Ex[ok_final] - E, wl.sigma_eV, wl.cutoff_sigmas).sum()
            expect = np.pi * E ** 2 * G / (2.0 * O.HBAR_EVS * P.Nq) * d
            assert abs(W[q, s] - expect) <= 1e-10 * expect, (q, s, W[q, s], expect)


def test_rates_are_point_group_invariant_on_the_two_atom_model():
    """W(S q) = W(q) branch by branch for the 48 operations on the 8-band / 2-atom drag model
    (6 branches, the two atoms with different g; q on a 4^3 mesh): each q is decomposed on its
    own by numpy, so the equality also needs the degenerate-group average."""
    wl = dataclasses.replace(S.workload_cscl8(4, 4), isotopes=(G, 3 * G))
    P = O.prepare(wl)
    W = O.isotope_rates(P, wl.isotopes)
    n = np.array(wl.qmesh)
    scale = W.max()
    for Sop in wl.model.sym_rot:
        img = O.flat_index(np.mod(P.qidx @ Sop.T, n), tuple(n))
        np.testing.assert_allclose(W[img], W, rtol=1e-9, atol=1e-12 * scale)


def test_flat_delta_limit_gives_the_atom_weights():
    """Completeness of the eigenvectors at every q': sum_s' |xi*_{tau,s} . xi_{tau,s'q'}|^2 =
    |xi_{tau,s}|^2.  With a delta flat across the phonon band (sigma = 10 eV: within 2e-5 over
    60 meV) and no mode left out, W(sq) = pi E^2 delta0 / (2 hbar) sum_tau g_tau |xi_{tau,sq}|^2,
    averaged over the degenerate group: the 2-atom model's two masses give the atoms different
    weights in every mode, and different g."""
    wl = dataclasses.replace(S.workload_cscl8(4, 4), isotopes=(G, 5 * G), sigma_eV=10.0, omega_min_eV=-1.0)
    with np.errstate(divide="ignore", invalid="ignore"):   # velocities of zero-frequency modes
        P = O.prepare(wl)
    W = O.isotope_rates(P, wl.isotopes)
    d0 = 1.0 / (wl.sigma_eV * np.sqrt(2.0 * np.pi))
    wt = np.stack([np.sum(np.abs(P.u[:, 3 * t:3 * t + 3, :]) ** 2, axis=1) for t in range(2)], axis=-1)
    raw = np.pi * P.w ** 2 * d0 / (2.0 * O.HBAR_EVS) * (wt @ np.array(wl.isotopes))
    for q in range(P.Nq):
        for grp in O.degenerate_groups(P.w[q], wl.degen_tol_eV):
            expect = raw[q, grp].mean()
            np.testing.assert_allclose(W[q, grp], expect, rtol=1e-4, atol=1e-12 * raw.max())
    assert np.ptp(wt[:, :, 0][P.w > 1e-3]) > 0.5      # the atoms' weights really differ


def test_rates_are_linear_in_the_mass_variance():
    P = O.prepare(_sc1(n=6))
    np.testing.assert_allclose(O.isotope_rates(P, (3 * G,)), 3 * O.isotope_rates(P, (G,)), rtol=1e-13)


def test_rta_rates_obey_matthiessens_rule_and_kappa_drops():
    """Eq. W^RTA_sq: the isotope rate adds to the e-ph and background ones mode by mode; the
    extra phonon scattering lowers the phonon thermal conductivity."""
    wl = _sc1()
    P = O.prepare(wl)
    R = O.transition_rates(P)
    with_iso = O.solve_coupled_bte(P, R, level="dragged")
    P0 = dataclasses.replace(P, wl=dataclasses.replace(wl, isotopes=None))
    without = O.solve_coupled_bte(P0, R, level="dragged")
    np.testing.assert_allclose(with_iso.W_ph - without.W_ph, O.isotope_rates(P, (G,)), rtol=1e-10,
                               atol=1e-12 * with_iso.W_ph.max())
    assert with_iso.coeffs["kappa_ph"][0, 0] < without.coeffs["kappa_ph"][0, 0]
