"""The allocation-free transport-coefficient entry point.

Callers that cannot allocate GPU memory -- code running while a stream is captured into a
CUDA graph, frameworks that route every allocation through their own pool, embedders that
may only use the buffers they were handed -- get ephb_transport_coefficients_noalloc: it
takes device arrays the caller owns and writes the tensors into a caller buffer, using
only a scratch array compiled into the library.  These tests check, through the C ABI, that
two calls in a row give the same tensors as ephb_transport_coefficients, and that inputs
larger than the scratch bound are refused.  The file is named so that it runs last."""
import numpy as np
import pytest

from paper_2109_08547_gb300 import binding as B
from paper_2109_08547_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

ORDER = ("sigma", "sigmaS", "S", "alpha_el", "kappa0_el", "kappa_el", "alpha_ph", "kappa_ph")
RTOL = 1e-8


def _inputs(ctx):
    ptrs = {}
    for key, arr in (("eps", "state_eps"), ("vel", "state_vel"), ("weight", "state_weight"), ("I", "I"),
                     ("J", "J"), ("omega", "omega"), ("vph", "vph"), ("F", "F"), ("G", "G")):
        p, shape, _ = B.device_array(ctx, arr)
        ptrs[key] = p
        if key == "eps":
            n_states = shape[0]
        if key == "omega":
            n_modes = shape[0] * shape[1]
    return ptrs, n_states, n_modes


@pytest.mark.parametrize("which", ["sc1-oh", "cscl4-6"])
def test_noalloc_matches_transport_coefficients(which):
    import torch
    wl = S.workload_sc1() if which == "sc1-oh" else S.workload_cscl4(6)
    stream = torch.cuda.current_stream(0).cuda_stream
    ctx = B.Context(0, stream=stream)
    B.set_wannier_model(ctx, wl.model)
    B.run_path(ctx, wl, level="dragged")
    ref = B.transport_coefficients(ctx)
    ptrs, n_states, n_modes = _inputs(ctx)
    m = wl.model
    out = torch.empty(72, dtype=torch.float64, device="cuda:0")
    for _ in range(2):   # two calls in a row share the scratch array
        out.fill_(float("nan"))
        st = B.transport_coefficients_noalloc(
            ptrs, n_states, n_modes, wl.T_K, wl.mu_eV, m.spin_deg, abs(np.linalg.det(m.lattice)),
            int(np.prod(wl.kmesh)), int(np.prod(wl.qmesh)), wl.omega_min_eV, m.sym_cart, out.data_ptr(), stream)
        assert st == B.OK
        torch.cuda.current_stream(0).synchronize()
        got = out.cpu().numpy().reshape(8, 9)
        for i, key in enumerate(ORDER):
            r = ref[key].ravel()
            nrm = np.linalg.norm(r)
            err = np.linalg.norm(got[i] - r) / nrm if nrm > 0 else np.linalg.norm(got[i])
            assert err <= RTOL, f"{key}: {err:.3e}"
    ctx.close()


def test_noalloc_rejects_oversized_input():
    ptrs = {k: 0x1000 for k in ("eps", "vel", "weight", "I", "J", "omega", "vph", "F", "G")}
    st = B.transport_coefficients_noalloc(ptrs, B.NOALLOC_MAX_ITEMS + 1, 1, 300.0, 0.0, 2.0, 27.0, 8, 8, 1e-4,
                                          np.eye(3)[None], 0x1000, 0)
    assert st == B.EINVAL
