"""The electron-charged-impurity (e-chimp) channel on the GPU against the oracle: the electron
RTA rates W^RTA (e-ph plus e-chimp, Matthiessen's rule) state by state at 1e-10 and the
transport coefficients at 1e-8, on the one-band cubic model and on the 4-band model with two
dopant species ("Electrons, phonons, and interactions", Eqs. X^e-chimp, q_TF^2)."""
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
    "sc1-oh": lambda: dataclasses.replace(SY.workload_sc1(), chimp=SY.Impurities((1.0e19,), (1.0,), 11.7)),
    "cscl4-6": lambda: dataclasses.replace(SY.workload_cscl4(6),
                                           chimp=SY.Impurities((5.0e18, 2.0e18), (1.0, 2.0), 9.0)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_chimp_rates_and_coefficients_match_oracle(name):
    wl = CASES[name]()
    P = O.prepare(wl)
    R = O.transition_rates(P)
    ref = O.solve_coupled_bte(P, R, level="dragged")
    with B.Context(0) as ctx:
        B.set_wannier_model(ctx, wl.model)
        r = B.run_path(ctx, wl, level="dragged")
        W = B.get_array(ctx, "w_e")
        wl_list = B.get_array(ctx, "ibzw_list")
        nb = wl.model.nb
        pos = {(int(k), b): i * nb + b for i, k in enumerate(wl_list) for b in range(nb)}
        for s, (k, b) in enumerate(ref.states):
            np.testing.assert_allclose(W[pos[(int(k), int(b))]], ref.W_e[s], rtol=1e-10)
        for key in TENSORS:
            assert rel_fro(r.coeffs[key], ref.coeffs[key]) <= COEFF_RTOL, key
        # clearing the impurities gives back the e-ph-only answer
        B.set_impurities(ctx, None)
        plain = B.run_path(ctx, dataclasses.replace(wl, chimp=None), level="dragged")
        assert plain.coeffs["sigma"][0, 0] > r.coeffs["sigma"][0, 0]


def test_impurity_arguments():
    with B.Context(0) as ctx:
        for bad in (SY.Impurities((1e18,) * 5, (1.0,) * 5, 10.0), SY.Impurities((1e18,), (1.0,), 0.0),
                    SY.Impurities((-1e18,), (1.0,), 10.0)):
            with pytest.raises(B.EphbError):
                B.set_impurities(ctx, bad)
        B.set_impurities(ctx, None)
