"""The phonon-isotope (Tamura) channel on the GPU against the oracle: the phonon RTA rates
W^RTA_sq (e-ph, background and isotope, Matthiessen's rule) mode by mode at 1e-10 and the
transport coefficients at 1e-8, on the one-band cubic model (Cartesian phonons, O_h wedge) and
on the 4-band, 2-atom model with a different g for each atom ("Electrons, phonons, and
interactions", Eq. W^ph-x)."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2109_08547_gb300 import binding as B
from paper_2109_08547_gb300 import synthetic as SY
from _parity import COEFF_RTOL, rel_fro

pytestmark = pytest.mark.gpu

TENSORS = ("sigma", "sigmaS", "alpha_el", "kappa0_el", "alpha_ph", "kappa_ph")
CASES = {
    "sc1-oh": lambda: dataclasses.replace(SY.workload_sc1(), isotopes=(2.0e-4,)),
    "cscl4-6": lambda: dataclasses.replace(SY.workload_cscl4(6), isotopes=(2.0e-4, 6.0e-4)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_isotope_rates_and_coefficients_match_oracle(name):
    wl = CASES[name]()
    P = O.prepare(wl)
    R = O.transition_rates(P)
    ref = O.solve_coupled_bte(P, R, level="dragged")
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        r = B.run_path(ctx, wl, level="dragged")
        W = B.get_array(ctx, "w_ph").reshape(ref.W_ph.shape)
        np.testing.assert_allclose(W, ref.W_ph, rtol=1e-10, atol=1e-12 * ref.W_ph.max())
        for key in TENSORS:
            assert rel_fro(r.coeffs[key], ref.coeffs[key]) <= COEFF_RTOL, key
        plain = B.run_path(ctx, dataclasses.replace(wl, isotopes=None), level="dragged")
        assert plain.coeffs["kappa_ph"][0, 0] > r.coeffs["kappa_ph"][0, 0]


def test_isotope_arguments():
    wl = SY.workload_sc1()
    with B.Context(0) as ctx:
        with pytest.raises(B.EphbError):
            B.set_isotopes(ctx, (1e-4,) * 5)
        with pytest.raises(B.EphbError):
            B.set_isotopes(ctx, (-1e-4,))
        B.set_wannier_model(ctx, wl.model)
        B.build_meshes_ibz(ctx, wl.kmesh, wl.qmesh, wl.window)
        B.compute_transition_rates(ctx, wl.T_K, wl.mu_eV)
        B.set_isotopes(ctx, (1e-4, 1e-4))   # two atoms for a one-atom model: refused at the solve
        with pytest.raises(B.EphbError):
            B.solve_coupled_bte(ctx, "dragged", 1e-10)
