"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and turn
its device arrays into the oracle's (k, m, q, n, s) keyed tables."""
import numpy as np

from paper_2109_08547_gb300 import binding as B

# tolerances (FP64 path)
RATE_RTOL = 1e-10          # per entry, relative, with a floor of 1e-6 * max |X|
RATE_FLOOR = 1e-6
COEFF_RTOL = 1e-8          # per tensor, relative Frobenius norm


def run_gpu(wl, level="dragged", ko=True, tol=None, ctx=None):
    ctx = ctx or B.Context(0)
    B.set_wannier_model(ctx, wl.model)
    res = B.run_path(ctx, wl, level=level, ko_correction=ko, tol=tol)
    return ctx, res


def gpu_rate_table(ctx, wl):
    """dict (ik, m, iq, n, s) -> (X+, X-) from the electron-side CSR."""
    nb = wl.model.nb
    ibzw = B.get_array(ctx, "ibzw_list")
    row_ptr = B.get_array(ctx, "row_ptr")
    kpns = B.get_array(ctx, "entry_kpns").astype(np.int64)
    X = B.get_array(ctx, "entry_x").reshape(-1, 2)
    kp = kpns & ((1 << 21) - 1)
    n = (kpns >> 21) & 15
    s = kpns >> 25
    nrow = len(row_ptr) - 1
    lens = np.diff(row_ptr)
    row = np.repeat(np.arange(nrow), lens)
    ik = ibzw[row // nb].astype(np.int64)
    m = row % nb
    km, qm = np.array(wl.kmesh), np.array(wl.qmesh)
    ratio = km // qm

    def coords(k):
        return np.stack([k // (km[1] * km[2]), (k // km[2]) % km[1], k % km[2]], axis=-1)

    d = np.mod(coords(kp) - coords(ik), km) // ratio
    iq = (d[:, 0] * qm[1] + d[:, 1]) * qm[2] + d[:, 2]
    return {(int(a), int(b), int(c), int(e), int(f)): (x0, x1)
            for a, b, c, e, f, x0, x1 in zip(ik, m, iq, n, s, X[:, 0], X[:, 1])}


def oracle_rate_table(R):
    return {(int(a), int(b), int(c), int(e), int(f)): (x0, x1)
            for a, b, c, e, f, x0, x1 in zip(R.ik, R.m, R.iq, R.n, R.s, R.Xp, R.Xm)}


def compare_rates(gpu, ora, P=None, rows=None):
    """Every oracle entry must be present with matching X+, X-; extra/missing keys are only
    allowed for tuples whose delta argument sits within 1e-9 eV of the cut."""
    if rows is not None:
        gpu = {k: v for k, v in gpu.items() if k[0] in rows}
    xmax = max(max(abs(v[0]), abs(v[1])) for v in ora.values())
    floor = RATE_FLOOR * xmax
    worst = 0.0
    for key, (xp, xm) in ora.items():
        assert key in gpu or (P is not None and _near_cut(P, key)), f"missing entry {key}"
        if key not in gpu:
            continue
        gp, gm = gpu[key]
        for a, b in ((gp, xp), (gm, xm)):
            err = abs(a - b) / max(abs(b), floor)
            worst = max(worst, err)
    extra = set(gpu) - set(ora)
    for key in extra:
        assert P is not None and _near_cut(P, key), f"unexpected entry {key}"
    assert worst <= RATE_RTOL, f"worst relative rate error {worst:.3e}"
    return worst


def _near_cut(P, key):
    ik, m, iq, n, s = key
    import oracle as O
    kp = O.kplusq(P, ik, np.array([iq]))[0]
    x = P.eps[kp, n] - P.eps[ik, m]
    cut = P.wl.cutoff_sigmas * P.wl.sigma_eV
    w = P.w[iq, s]
    return min(abs(abs(x - w) - cut), abs(abs(x + w) - cut)) < 1e-9


def rel_fro(a, b):
    nb = np.linalg.norm(b)
    if nb == 0:
        return np.linalg.norm(a)
    return np.linalg.norm(a - b) / nb
