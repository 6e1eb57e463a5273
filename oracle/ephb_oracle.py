"""FP64 CPU oracle (test infrastructure only; see the package docstring).

Plain, slow, readable double-precision restatement of arXiv 2109.08547:
  * Wannier-to-Bloch interpolation of H, D and g            (Eqs. H_mn(k), D_ss'(q), g^smn_kq)
  * Hellmann-Feynman electron and phonon velocities         (Eqs. v_mk, v_sq)
  * e-ph transition rates X^+ / X^- over IBZ k x FBZ k'     (Eq. X^e-ph)
  * e-chimp rates (screened Coulomb, Born)                  (Eqs. |g^e-chimp_q|^2, q_TF^2, X^e-chimp)
  * ph-isotope rates (Tamura)                               (Eq. W^ph-x)
  * ph-e rates Y (the same + process seen from the phonon)  (Eq. Y^ph-e)
  * RTA terms and rates, self and drag terms                (Eqs. I0/J0, W^RTA, dI^S, dI^D, F0/G0, dF^D)
  * unified single-iterator coupled solution                ("Coupled and decoupled BTEs")
  * Kelvin-Onsager correction                               (Eqs. sigmaS = alpha/T, I = I_diff + I_drag)
  * transport coefficients                                  (Eqs. sigma/sigmaS, alpha_el/kappa0_el, alpha_ph/kappa_ph)

Readings of passages the paper leaves silent or garbled (each also listed in the
design notes): Wigner-Seitz weights and 1/N factors absorbed into the Wannier
arrays; g prefactor sqrt(w_ref/w_sq) with the mass inside the Cartesian sum;
|g|^2 and velocities averaged over degenerate subspaces; Gaussian delta with an
8-sigma cut; modes with hbar*w < omega_min excluded; X normalised by 1/N_q and Y by
1/N_k; phonon background rate W_bg replacing ph-ph scattering; Jacobi
iteration without mixing; residual = max relative Frobenius change of the
coefficient tensors; Kelvin-Onsager scalar by least squares; coefficient sums
carry 1/N_k and 1/N_q.
"""
from __future__ import annotations

import dataclasses

import numpy as np

HBAR_EVS = 6.582119569e-16     # eV s
KB_EVK = 8.617333262e-5        # eV / K
E_CHARGE = 1.602176634e-19     # C
ANGSTROM = 1.0e-10             # m

__all__ = [
    "HBAR_EVS", "KB_EVK", "E_CHARGE", "mesh_indices", "flat_index", "degenerate_groups",
    "electron_bands", "phonon_modes", "irreducible_wedge", "bloch_vertex_sq",
    "transition_rates", "Rates", "BTEResult", "solve_coupled_bte", "coefficients_from_responses",
    "prepare", "Prepared", "gaussian_delta", "fermi", "bose", "StateSpace", "ibz_window_points",
    "kplusq", "minus_q", "TENSORS", "inverse_ops", "ANGSTROM", "ibz_window_rows", "prepare_rows",
    "tetra_corner_weights", "tetra_point_weights", "CUBE_TETRAHEDRA", "CUBE_SUBDIVISIONS",
    "EPS0", "centred", "reciprocal_si", "thomas_fermi_q2", "chimp_g2", "chimp_kernel", "chimp_rates",
    "isotope_rates",
]


# ----------------------------------------------------------------------------------------
# meshes and degeneracies
# ----------------------------------------------------------------------------------------

def mesh_indices(n) -> np.ndarray:
    """Gamma-centred mesh, point index (i0*n1 + i1)*n2 + i2, crystal coords i/n."""
    i0, i1, i2 = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    return np.stack([i0.ravel(), i1.ravel(), i2.ravel()], axis=1).astype(np.int64)


def flat_index(idx: np.ndarray, n) -> np.ndarray:
    return (idx[..., 0] * n[1] + idx[..., 1]) * n[2] + idx[..., 2]


def degenerate_groups(e: np.ndarray, tol: float) -> list:
    """Chains of consecutive (ascending) eigenvalues closer than tol."""
    groups, start = [], 0
    for i in range(1, len(e) + 1):
        if i == len(e) or e[i] - e[i - 1] >= tol:
            groups.append(np.arange(start, i))
            start = i
    return groups


def _group_average_matrix(e: np.ndarray, tol: float) -> np.ndarray:
    n = len(e)
    A = np.zeros((n, n))
    for grp in degenerate_groups(e, tol):
        A[np.ix_(grp, grp)] = 1.0 / len(grp)
    return A


# ----------------------------------------------------------------------------------------
# electrons and phonons (Eqs. H_mn(k), v_mk, D_ss'(q), v_sq)
# ----------------------------------------------------------------------------------------

def electron_bands(model, kcrys: np.ndarray, degen_tol: float):
    """H(k) = sum_Re exp(i k.Re) H(Re); eigenvalues eps_mk (ascending), eigenvector
    columns c (the paper's U_k is c^dagger); v_mk = (1/hbar) <mk| grad_k H |mk>,
    averaged over degenerate subspaces.  Returns eps (eV), c, v (m/s)."""
    phase = np.exp(2j * np.pi * (kcrys @ model.Re.T.astype(np.float64)))
    Hk = np.einsum("kr,rmn->kmn", phase, model.H_R)
    eps, c = np.linalg.eigh(Hk)
    Rcart = model.Re.astype(np.float64) @ model.lattice
    vdiag = np.empty(eps.shape + (3,))
    for a in range(3):
        dH = np.einsum("kr,rmn->kmn", phase * (1j * Rcart[:, a])[None, :], model.H_R)
        vdiag[..., a] = np.einsum("kim,kij,kjm->km", c.conj(), dH, c).real
    for k in range(eps.shape[0]):
        vdiag[k] = _group_average_matrix(eps[k], degen_tol) @ vdiag[k]
    return eps, c, vdiag * (ANGSTROM / HBAR_EVS)


def phonon_modes(model, qcrys: np.ndarray, degen_tol: float, omega_min: float):
    """D(q) = sum_Rph exp(i q.Rph) D(Rph) (mass scaled, eV^2); hbar*w = sqrt(eigenvalue)
    (negative eigenvalues clipped to 0); v_sq = (1/hbar)(1/(2 hbar w)) <sq|grad_q D|sq>,
    the matrix element averaged over degenerate subspaces; v = 0 for modes below
    omega_min.  Returns w (eV), u, v (m/s)."""
    phase = np.exp(2j * np.pi * (qcrys @ model.Rd.T.astype(np.float64)))
    Dq = np.einsum("qr,rab->qab", phase, model.D_R)
    lam, u = np.linalg.eigh(Dq)
    w = np.sqrt(np.maximum(lam, 0.0))
    Rcart = model.Rd.astype(np.float64) @ model.lattice
    vdiag = np.empty(w.shape + (3,))
    for a in range(3):
        dD = np.einsum("qr,rab->qab", phase * (1j * Rcart[:, a])[None, :], model.D_R)
        vdiag[..., a] = np.einsum("qis,qij,qjs->qs", u.conj(), dD, u).real
    v = np.zeros_like(vdiag)
    for q in range(w.shape[0]):
        avg = _group_average_matrix(w[q], degen_tol) @ vdiag[q]
        ok = w[q] > omega_min
        v[q, ok] = avg[ok] / (2.0 * w[q, ok, None])
    return w, u, v * (ANGSTROM / HBAR_EVS)


# ----------------------------------------------------------------------------------------
# symmetry: irreducible wedge of the k mesh
# ----------------------------------------------------------------------------------------

def irreducible_wedge(n, sym_rot: np.ndarray):
    """For every mesh point k: representative <k> = smallest flat index among the images
    S k, the first operation (in list order) with S <k> = k, and the stabiliser size of
    <k>.  Also returns the index table of the image of every point under every S."""
    idx = mesh_indices(n)
    nn = np.array(n)
    images = np.stack([flat_index(np.mod(idx @ S.T.astype(np.int64), nn), n) for S in sym_rot])
    rep = images.min(axis=0)
    N = idx.shape[0]
    op = np.empty(N, dtype=np.int64)
    stab = np.empty(N, dtype=np.int64)
    for k in range(N):
        r = rep[k]
        op[k] = int(np.nonzero(images[:, r] == k)[0][0])
        stab[k] = int(np.count_nonzero(images[:, r] == r))
    return rep, op, stab, images


def inverse_ops(sym_rot: np.ndarray) -> np.ndarray:
    inv = np.empty(len(sym_rot), dtype=np.int64)
    for i, S in enumerate(sym_rot):
        Si = np.rint(np.linalg.inv(S)).astype(np.int64)
        inv[i] = [j for j, T in enumerate(sym_rot) if np.array_equal(T, Si)][0]
    return inv


# ----------------------------------------------------------------------------------------
# occupations and delta
# ----------------------------------------------------------------------------------------

def fermi(e, mu, T):
    return 1.0 / (np.exp((e - mu) / (KB_EVK * T)) + 1.0)


def bose(w, T):
    out = np.zeros_like(w)
    ok = w > 0
    out[ok] = 1.0 / np.expm1(w[ok] / (KB_EVK * T))
    return out


def gaussian_delta(x, sigma, cutoff):
    """delta(x) = exp(-x^2/(2 sigma^2)) / (sigma sqrt(2 pi)); exactly 0 beyond cutoff*sigma."""
    d = np.exp(-0.5 * (x / sigma) ** 2) / (sigma * np.sqrt(2.0 * np.pi))
    return np.where(np.abs(x) <= cutoff * sigma, d, 0.0)


# ----------------------------------------------------------------------------------------
# linear tetrahedron delta ("Workflow and structure": the analytic tetrahedron method)
# ----------------------------------------------------------------------------------------

# The six tetrahedra of a mesh cube around one of its body diagonals (corner c has the offset
# (c&1, c>>1&1, c>>2&1)): the diagonal 0-7 and its images a^c, a = 1, 2, 4, for the other three.
# One diagonal's subdivision is not invariant under the cubic group; the average over the four
# is (reading [A22]).
CUBE_TETRAHEDRA = ((0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7), (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 6, 7))
CUBE_SUBDIVISIONS = tuple(tuple(tuple(a ^ c for c in tet) for tet in CUBE_TETRAHEDRA) for a in (0, 1, 2, 4))


def tetra_corner_weights(e, E):
    """Delta weights of the four corners of one tetrahedron: W_c = (1/V) int_T delta(E - e(r)) lam_c(r) dr
    for e linear in the barycentric coordinates lam (e(r) = sum_c lam_c(r) e_c).  The level set
    e = E is a triangle or a quadrilateral whose vertices lie on the edges (i, j) with
    e_i < E < e_j; int_S lam_c dA / |grad e| over it, with the reference simplex of volume 1/6 in
    the coordinates (lam_2, lam_3, lam_4) of the corners sorted by energy.  Zero unless
    e_min < E < e_max."""
    e = np.asarray(e, dtype=np.float64)
    order = np.argsort(e, kind="stable")
    es = e[order]
    W = np.zeros(4)
    if not (es[0] < E < es[3]):
        return W
    if E < es[1]:
        edges = ((0, 1), (0, 2), (0, 3))
    elif E < es[2]:
        edges = ((0, 2), (0, 3), (1, 3), (1, 2))
    else:
        edges = ((0, 3), (1, 3), (2, 3))
    pts = []
    for i, j in edges:
        t = (E - es[i]) / (es[j] - es[i])
        lam = np.zeros(4)
        lam[i], lam[j] = 1.0 - t, t
        pts.append(lam)
    tris = [(0, 1, 2)] if len(pts) == 3 else [(0, 1, 2), (0, 2, 3)]
    grad = np.array([es[1] - es[0], es[2] - es[0], es[3] - es[0]])
    acc = np.zeros(4)
    for a, b, c in tris:
        x = [pts[a][1:], pts[b][1:], pts[c][1:]]
        area = 0.5 * np.linalg.norm(np.cross(x[1] - x[0], x[2] - x[0]))
        acc += area * (pts[a] + pts[b] + pts[c]) / 3.0
    W[order] = acc / (np.linalg.norm(grad) / 6.0)
    return W


def _tetra_weights_batch(e, corner):
    """tetra_corner_weights for many tetrahedra at E = 0, the weight of one corner each:
    e (m, 4) corner values, corner (m,) the corner's position in e.  Same construction, array
    by array: the three energy ranges are evaluated for every tetrahedron and selected."""
    m = e.shape[0]
    order = np.argsort(e, axis=1, kind="stable")
    es = np.take_along_axis(e, order, axis=1)
    pc = np.argmax(order == corner[:, None], axis=1)           # sorted position of the corner
    out = np.zeros(m)
    cases = (((0, 1), (0, 2), (0, 3)), ((0, 2), (0, 3), (1, 3), (1, 2)), ((0, 3), (1, 3), (2, 3)))
    sel = [(0.0 < es[:, 1]), (es[:, 1] <= 0.0) & (0.0 < es[:, 2]), (es[:, 2] <= 0.0)]
    valid = (es[:, 0] < 0.0) & (0.0 < es[:, 3])
    gnorm = np.linalg.norm(es[:, 1:] - es[:, :1], axis=1)
    for edges, mask in zip(cases, sel):
        rows = np.nonzero(valid & mask)[0]
        if len(rows) == 0:
            continue
        esr = es[rows]
        lam = np.zeros((len(rows), len(edges), 4))
        for p, (i, j) in enumerate(edges):
            t = (0.0 - esr[:, i]) / (esr[:, j] - esr[:, i])
            lam[:, p, i] = 1.0 - t
            lam[:, p, j] = t
        lc = lam[np.arange(len(rows)), :, pc[rows]]                 # (r, npts): lambda of the corner
        x = lam[:, :, 1:]
        tris = [(0, 1, 2)] if len(edges) == 3 else [(0, 1, 2), (0, 2, 3)]
        acc = np.zeros(len(rows))
        for a, b, c in tris:
            area = 0.5 * np.linalg.norm(np.cross(x[:, b] - x[:, a], x[:, c] - x[:, a]), axis=1)
            acc += area * (lc[:, a] + lc[:, b] + lc[:, c]) / 3.0
        out[rows] = acc / (gnorm[rows] / 6.0)
    return out


def tetra_point_weights(values, n, pts):
    """w(p) = (1 / (6 N)) sum over the tetrahedra containing mesh point p of p's corner weight at
    E = 0, averaged over the four body-diagonal subdivisions of the mesh cubes, for a function
    `values` on the n1 x n2 x n3 mesh linearly interpolated in every tetrahedron
    (sum_p w(p) F(p) approximates the zone average of F delta(values))."""
    nn = np.array(n)
    N = int(np.prod(nn))
    vals = np.asarray(values).reshape(N)
    pts = np.asarray(pts, dtype=np.int64)
    idx = mesh_indices(n)
    # every (point, cube it is a corner of, subdivision, tetrahedron holding that corner)
    combos = []
    for cb in range(8):
        shift = np.array([cb & 1, (cb >> 1) & 1, (cb >> 2) & 1])
        for sub in CUBE_SUBDIVISIONS:
            for tet in sub:
                if cb in tet:
                    combos.append((shift, tet, tet.index(cb)))
    out = np.zeros(len(pts))
    for shift, tet, pos in combos:
        origin = idx[pts] - shift
        corners = np.stack([flat_index(np.mod(origin + np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1]), nn), n)
                            for c in tet], axis=1)
        out += 0.25 * _tetra_weights_batch(vals[corners], np.full(len(pts), pos))
    return out / (6.0 * N)


# ----------------------------------------------------------------------------------------
# prepared state: bands on the full k mesh, phonons on the full q mesh, windows, IBZ
# ----------------------------------------------------------------------------------------

@dataclasses.dataclass
class Prepared:
    wl: object
    kidx: np.ndarray
    qidx: np.ndarray
    eps: np.ndarray
    c: np.ndarray
    vel: np.ndarray
    w: np.ndarray
    u: np.ndarray
    vph: np.ndarray
    active: np.ndarray        # (Nk, nb) bool
    rep: np.ndarray
    op: np.ndarray
    stab: np.ndarray
    ratio: np.ndarray         # k mesh = ratio * q mesh, per dimension
    inv_op: np.ndarray
    qimages: np.ndarray       # (nsym, Nq) image of q under S

    @property
    def Nk(self):
        return self.kidx.shape[0]

    @property
    def Nq(self):
        return self.qidx.shape[0]


def prepare(wl) -> Prepared:
    m = wl.model
    kidx = mesh_indices(wl.kmesh)
    qidx = mesh_indices(wl.qmesh)
    eps, c, vel = electron_bands(m, kidx / np.array(wl.kmesh, dtype=np.float64), wl.degen_tol_eV)
    w, u, vph = phonon_modes(m, qidx / np.array(wl.qmesh, dtype=np.float64), wl.degen_tol_eV, wl.omega_min_eV)
    lo, hi = wl.window
    active = (eps >= lo) & (eps <= hi)
    rep, op, stab, _ = irreducible_wedge(wl.kmesh, m.sym_rot)
    ratio = np.array(wl.kmesh) // np.array(wl.qmesh)
    qq = np.array(wl.qmesh)
    qimages = np.stack([flat_index(np.mod(qidx @ S.T.astype(np.int64), qq), wl.qmesh) for S in m.sym_rot])
    return Prepared(wl=wl, kidx=kidx, qidx=qidx, eps=eps, c=c, vel=vel, w=w, u=u, vph=vph, active=active,
                    rep=rep, op=op, stab=stab, ratio=ratio, inv_op=inverse_ops(m.sym_rot), qimages=qimages)


def ibz_window_rows(wl) -> np.ndarray:
    """The irreducible representatives (smallest flat index of each star) holding an active
    band, from bands computed on the representatives only (large meshes)."""
    kidx = mesh_indices(wl.kmesh)
    nn = np.array(wl.kmesh)
    images = np.stack([flat_index(np.mod(kidx @ S.T.astype(np.int64), nn), wl.kmesh) for S in wl.model.sym_rot])
    reps = np.unique(images.min(axis=0))
    lo, hi = wl.window
    act = np.zeros(len(reps), bool)
    for c0 in range(0, len(reps), 65536):
        e, _, _ = electron_bands(wl.model, kidx[reps[c0:c0 + 65536]] / nn, wl.degen_tol_eV)
        act[c0:c0 + 65536] = ((e >= lo) & (e <= hi)).any(axis=1)
    return reps[act]


def prepare_rows(wl, rows) -> Prepared:
    """A Prepared state for transition_rates(P, ks=rows) on a large mesh: bands, eigenvectors
    and velocities only at the given k rows and their partners k + q (zero elsewhere, never
    read by the rates of those rows); phonons on the whole q mesh.  The symmetry tables are
    not filled (the rates of given rows do not use them)."""
    kidx = mesh_indices(wl.kmesh)
    qidx = mesh_indices(wl.qmesh)
    nk, nq = np.array(wl.kmesh), np.array(wl.qmesh)
    ratio = nk // nq
    need = [np.asarray(rows, dtype=np.int64)]
    for k in rows:
        need.append(flat_index(np.mod(kidx[k][None, :] + ratio[None, :] * qidx, nk), wl.kmesh))
    need = np.unique(np.concatenate(need))
    nb = wl.model.nb
    eps = np.zeros((kidx.shape[0], nb))
    c = np.zeros((kidx.shape[0], nb, nb), dtype=np.complex128)
    vel = np.zeros((kidx.shape[0], nb, 3))
    for c0 in range(0, len(need), 65536):
        sel = need[c0:c0 + 65536]
        eps[sel], c[sel], vel[sel] = electron_bands(wl.model, kidx[sel] / nk, wl.degen_tol_eV)
    w, u, vph = phonon_modes(wl.model, qidx / nq, wl.degen_tol_eV, wl.omega_min_eV)
    lo, hi = wl.window
    active = np.zeros(eps.shape, dtype=bool)
    active[need] = (eps[need] >= lo) & (eps[need] <= hi)
    none = np.full(kidx.shape[0], -1, dtype=np.int64)
    return Prepared(wl=wl, kidx=kidx, qidx=qidx, eps=eps, c=c, vel=vel, w=w, u=u, vph=vph, active=active,
                    rep=none, op=none, stab=none, ratio=ratio, inv_op=inverse_ops(wl.model.sym_rot),
                    qimages=None)


def kplusq(P: Prepared, k: int, q: np.ndarray) -> np.ndarray:
    """k' = [k + q] on the k mesh (q points of the phonon mesh, scaled by the mesh ratio)."""
    kk = np.array(P.wl.kmesh)
    return flat_index(np.mod(P.kidx[k][None, :] + P.ratio[None, :] * P.qidx[q], kk), P.wl.kmesh)


def minus_q(P: Prepared, q: np.ndarray) -> np.ndarray:
    return flat_index(np.mod(-P.qidx[q], np.array(P.wl.qmesh)), P.wl.qmesh)


# ----------------------------------------------------------------------------------------
# Bloch vertex (Eq. g^smn_kq)
# ----------------------------------------------------------------------------------------

def bloch_vertex_sq(P: Prepared, k: int, qs: np.ndarray, kps: np.ndarray) -> np.ndarray:
    """|g^s_mn(k,q)|^2 for one k and a list of q (k' = [k+q]), all bands and branches.

    g^s_mn = sqrt(w_ref / w_sq) sum_{m'n'alpha} c*_{n'n}(k') c_{m'm}(k)
             [ sum_{Re,Rp} exp(i k.Re + i q.Rp) gW_{m'n'alpha}(Re,Rp) ] u_{alpha s}(q) / sqrt(m_alpha/m_bar)

    The Fourier factor is the direct double sum over the pair (Re, Rp), written as a
    matrix product over the combined index.  |g|^2 is then averaged over the degenerate
    subspaces of the bands at k, the bands at k' and the branches at q.  Modes with
    hbar*w <= omega_min get |g|^2 = 0."""
    wl = P.wl
    m = wl.model
    nb, nbr = m.nb, m.nbranch
    kc = P.kidx[k] / np.array(wl.kmesh, dtype=np.float64)
    qc = P.qidx[qs] / np.array(wl.qmesh, dtype=np.float64)
    pe = kc @ m.Rge.T.astype(np.float64)                            # (nRe,)
    pp = qc @ m.Rgp.T.astype(np.float64)                            # (nq, nRp)
    phase = np.exp(2j * np.pi * (pe[None, :, None] + pp[:, None, :]))  # (nq, nRe, nRp)
    nRe, nRp = m.Rge.shape[0], m.Rgp.shape[0]
    G = phase.reshape(len(qs), nRe * nRp) @ m.g_R.reshape(nRe * nRp, nb * nb * nbr)
    G = G.reshape(len(qs), nb, nb, nbr)                              # [q, m', n', alpha]
    mass = np.repeat(m.mass_amu, 3)
    mscale = 1.0 / np.sqrt(mass / m.mass_amu.mean())
    w = P.w[qs]
    pref = np.zeros_like(w)
    ok = w > wl.omega_min_eV
    pref[ok] = np.sqrt(m.omega_ref_eV / w[ok])
    ck = P.c[k]                                                     # [m', m]
    ckp = P.c[kps]                                                  # [q, n', n]
    uq = P.u[qs] * mscale[None, :, None]                            # [q, alpha, s]
    g = np.einsum("am,qbn,qabx,qxs->qmns", ck, ckp.conj(), G, uq) * pref[:, None, None, :]
    g2 = np.abs(g) ** 2
    Ak = _group_average_matrix(P.eps[k], wl.degen_tol_eV)
    out = np.empty_like(g2)
    for i in range(len(qs)):
        Akp = _group_average_matrix(P.eps[kps[i]], wl.degen_tol_eV)
        Aq = _group_average_matrix(P.w[qs[i]], wl.degen_tol_eV)
        out[i] = np.einsum("ma,nb,sc,abc->mns", Ak, Akp, Aq, g2[i])
    return out


# ----------------------------------------------------------------------------------------
# transition rates (Eq. X^e-ph; Y^ph-e is the + process with the other normalisation)
# ----------------------------------------------------------------------------------------

@dataclasses.dataclass
class Rates:
    ik: np.ndarray      # full index of the IBZ representative (initial k)
    m: np.ndarray
    iq: np.ndarray
    n: np.ndarray
    s: np.ndarray
    ikp: np.ndarray     # full index of k' = [k + q]
    Xp: np.ndarray      # absorption rate X^+ (1/s)
    Xm: np.ndarray      # emission rate X^- (1/s)
    n_tuples: int       # (k m, q, n, s) tuples interpolated and delta-weighted
    n_pairs: int
    ibz_win: np.ndarray  # IBZ representatives with at least one active band


def ibz_window_points(P: Prepared) -> np.ndarray:
    reps = np.unique(P.rep)
    return np.array([k for k in reps if P.active[k].any()], dtype=np.int64)


def transition_rates(P: Prepared, ks=None, q_chunk: int = 256) -> Rates:
    """X^{+/-}_{m<k> n k'|sq} = (2 pi / (hbar N_q)) |g|^2 f_mk (1 - f_nk') {n_sq, 1 + n_sq}
    delta(eps_nk' - eps_mk -/+ hbar w_sq) for every IBZ representative <k> with an active
    band, every q of the phonon mesh with k' = [<k> + q] holding an active band, and every
    branch above omega_min.  Gaussian delta: an entry is kept when either delta argument lies
    within the cut.  Tetrahedron delta: (1/N_q) delta is replaced by the weight of q in the
    linear tetrahedron integral over the q mesh of delta(eps_n(<k>+q) - eps_mk -/+ w_s(q)), and an
    entry is kept when either weight is positive.  ``ks`` restricts the rows to a subset of IBZ
    representatives (sampling)."""
    wl = P.wl
    nb, nbr = wl.model.nb, wl.model.nbranch
    T, mu = wl.T_K, wl.mu_eV
    sig, cut = wl.sigma_eV, wl.cutoff_sigmas
    C = 2.0 * np.pi / (HBAR_EVS * P.Nq)
    fk = fermi(P.eps, mu, T)
    nq = bose(P.w, T)
    ibzw = ibz_window_points(P)
    rows = ibzw if ks is None else np.asarray(ks, dtype=np.int64)
    cols = {key: [] for key in ("ik", "m", "iq", "n", "s", "ikp", "Xp", "Xm")}
    n_tuples = 0
    n_pairs = 0
    allq = np.arange(P.Nq)
    tetra = getattr(wl, "delta", "gauss") == "tetra"
    for k in rows:
        kps_all = kplusq(P, k, allq)
        sel = P.active[kps_all].any(axis=1)
        qs_k = allq[sel]
        n_pairs += len(qs_k)
        if tetra:
            # weights of every pair q of the row, per (m, n, s, +/-): the zone integral over q of
            # delta(eps_n(k+q) - eps_m(k) -/+ w_s(q)), linear in every tetrahedron of the q mesh
            # (modes at or below omega_min enter with w = 0)
            tw = {}
            ws_all = np.where(P.w > wl.omega_min_eV, P.w, 0.0)
            for mm in np.nonzero(P.active[k])[0]:
                for nn in range(nb):
                    base = P.eps[kps_all, nn] - P.eps[k, mm]
                    for s in range(nbr):
                        tw[(mm, nn, s)] = (tetra_point_weights(base - ws_all[:, s], wl.qmesh, qs_k) * P.Nq,
                                           tetra_point_weights(base + ws_all[:, s], wl.qmesh, qs_k) * P.Nq)
            qpos = {int(q): j for j, q in enumerate(qs_k)}
        for c0 in range(0, len(qs_k), q_chunk):
            qs = qs_k[c0:c0 + q_chunk]
            kps = kps_all[qs]
            g2 = bloch_vertex_sq(P, k, qs, kps)
            for i, (q, kp) in enumerate(zip(qs, kps)):
                for mm in np.nonzero(P.active[k])[0]:
                    for nn in np.nonzero(P.active[kp])[0]:
                        for s in range(nbr):
                            if P.w[q, s] <= wl.omega_min_eV:
                                continue
                            n_tuples += 1
                            if tetra:
                                wpa, wma = tw[(mm, nn, s)]
                                dp, dm = wpa[qpos[int(q)]], wma[qpos[int(q)]]
                                if dp <= 0.0 and dm <= 0.0:
                                    continue
                            else:
                                xp = P.eps[kp, nn] - P.eps[k, mm] - P.w[q, s]
                                xm = P.eps[kp, nn] - P.eps[k, mm] + P.w[q, s]
                                if abs(xp) > cut * sig and abs(xm) > cut * sig:
                                    continue
                                dp, dm = gaussian_delta(xp, sig, cut), gaussian_delta(xm, sig, cut)
                            occ = C * g2[i, mm, nn, s] * fk[k, mm] * (1.0 - fk[kp, nn])
                            cols["ik"].append(k)
                            cols["m"].append(mm)
                            cols["iq"].append(q)
                            cols["n"].append(nn)
                            cols["s"].append(s)
                            cols["ikp"].append(kp)
                            cols["Xp"].append(occ * nq[q, s] * dp)
                            cols["Xm"].append(occ * (1.0 + nq[q, s]) * dm)
    arr = {key: np.array(v, dtype=np.float64 if key in ("Xp", "Xm") else np.int64) for key, v in cols.items()}
    order = np.lexsort((arr["s"], arr["n"], arr["iq"], arr["m"], arr["ik"]))
    arr = {key: v[order] for key, v in arr.items()}
    return Rates(n_tuples=n_tuples, n_pairs=n_pairs, ibz_win=ibzw, **arr)


# ----------------------------------------------------------------------------------------
# coupled BTE ("Coupled and decoupled BTEs") and coefficients ("Transport coefficients")
# ----------------------------------------------------------------------------------------

TENSORS = ("sigma", "sigmaS", "alpha_el", "kappa0_el", "alpha_ph", "kappa_ph")


# ----------------------------------------------------------------------------------------
# electron-charged-impurity scattering (e-chimp): Eqs. |g^e-chimp_q|^2, q_TF^2, X^e-chimp
# ----------------------------------------------------------------------------------------

EPS0 = 8.8541878128e-12        # F / m


def centred(frac: np.ndarray) -> np.ndarray:
    """Crystal coordinates reduced to [-1/2, 1/2) (for a cubic lattice: the nearest zone centre)."""
    return frac - np.floor(frac + 0.5)


def reciprocal_si(lattice_A: np.ndarray) -> np.ndarray:
    """Reciprocal lattice vectors (rows, 1/m) of lattice vectors given as rows in Angstrom."""
    return 2.0 * np.pi * np.linalg.inv(lattice_A).T / ANGSTROM


def thomas_fermi_q2(P: Prepared, imp) -> float:
    """Squared Thomas-Fermi wave vector (1/m^2), Eq. q_TF^2:
    d_s e^2 beta / (N_k V eps0 eps) sum_{mk} f(1 - f), over every band on the full k mesh."""
    wl = P.wl
    m = wl.model
    V = abs(np.linalg.det(m.lattice)) * ANGSTROM ** 3
    f = fermi(P.eps, wl.mu_eV, wl.T_K)
    beta = 1.0 / (KB_EVK * E_CHARGE * wl.T_K)          # 1/J
    return m.spin_deg * E_CHARGE ** 2 * beta * float(np.sum(f * (1.0 - f))) / (P.Nk * V * EPS0 * imp.eps_r)


def chimp_g2(q2: np.ndarray, q_tf2: float, imp, V: float) -> np.ndarray:
    """|g^e-chimp_q|^2 (eV^2) for squared wave vectors q2 (1/m^2), Eq. |g^e-chimp_q|^2:
    (1/V) sum_i n_i [Z_i e / (eps0 eps (q^2 + q_TF^2))]^2.  The bracket is in V m^3; with n_i in
    1/m^3 and V the cell volume in m^3 the result is in V^2, numerically eV^2 per carrier charge."""
    out = np.zeros_like(q2, dtype=np.float64)
    for n, Z in zip(imp.n_cm3, imp.Z):
        out = out + (n * 1e6) * (Z * E_CHARGE / (EPS0 * imp.eps_r * (q2 + q_tf2))) ** 2
    return out / V


def chimp_kernel(P: Prepared, states: np.ndarray):
    """Elastic e-chimp rates of Eq. X^e-chimp divided by the initial state's f(1 - f):
    K[a, b] = 2 pi / (hbar N_k) |g_q|^2 (1 - k.k' / (k k')) delta(eps_b - eps_a)
    for the initial states a = (k, m) (rows of `states`) and every active final state
    b = (k', n) of the full k mesh, q = [k' - k].  Readings: k, k' and q are Cartesian vectors of
    the centred crystal coordinates; a zero-length k or k' has transport factor 1; the final
    states are those of the window, as for the e-ph rates; delta is the e-ph Gaussian.
    Returns (K, final k indices, final bands)."""
    wl = P.wl
    m = wl.model
    imp = wl.chimp
    V = abs(np.linalg.det(m.lattice)) * ANGSTROM ** 3
    Bm = reciprocal_si(m.lattice)
    frac = P.kidx / np.array(wl.kmesh, dtype=np.float64)
    kc = centred(frac) @ Bm
    fk, fb = np.nonzero(P.active)
    ka, ma = states[:, 0], states[:, 1]
    dq = centred(frac[fk][None, :, :] - frac[ka][:, None, :]) @ Bm
    g2 = chimp_g2(np.sum(dq * dq, axis=-1), thomas_fermi_q2(P, imp), imp, V)
    na = np.linalg.norm(kc[ka], axis=1)
    nb = np.linalg.norm(kc[fk], axis=1)
    den = na[:, None] * nb[None, :]
    cos = np.where(den > 0.0, (kc[ka] @ kc[fk].T) / np.where(den > 0.0, den, 1.0), 0.0)
    cos = np.clip(cos, -1.0, 1.0)   # rounding must not make 1 - cos (k' = k: zero) negative
    delta = gaussian_delta(P.eps[fk, fb][None, :] - P.eps[ka, ma][:, None], wl.sigma_eV, wl.cutoff_sigmas)
    K = 2.0 * np.pi / (HBAR_EVS * P.Nk) * g2 * (1.0 - cos) * delta
    return K, fk, fb


def chimp_rates(P: Prepared, states: np.ndarray) -> np.ndarray:
    """The e-chimp part of W^RTA of each state (Eq. W^RTA_mk, Matthiessen's rule):
    sum_{nk'} X^e-chimp / (f (1 - f))."""
    K, _, _ = chimp_kernel(P, states)
    return K.sum(axis=1)


# ----------------------------------------------------------------------------------------
# phonon-isotope scattering (Tamura): Eq. W^ph-x and its entry into W^RTA_sq
# ----------------------------------------------------------------------------------------

def isotope_rates(P: Prepared, g_atoms) -> np.ndarray:
    """The ph-isotope part of W^RTA_sq (Eq. W^ph-x summed over s'q' and divided by n(1+n)), on the
    full q mesh: pi w_sq^2 / (2 N_q) sum_tau g_tau sum_{s'q'} |xi*_{tau,sq} . xi_{tau,s'q'}|^2
    delta(w_s'q' - w_sq).  With energies E = hbar w in eV and delta(w) = hbar delta(E) this is
    pi E^2 / (2 hbar N_q) sum ... delta(E' - E).  Readings: the printed rate carries no 1/N_q,
    which a mesh sum needs (as X^e-ph does); modes at or below omega_min take no part, on either
    side; delta is the e-ph Gaussian; the rate is averaged over the degenerate group of sq (the
    gauge inside a degenerate subspace is arbitrary).  g_atoms: mass-variance parameter g_tau of
    each atom of the basis."""
    wl = P.wl
    w, u = P.w, P.u
    Nq, nbr = w.shape
    ok = w > wl.omega_min_eV
    ov = np.zeros((Nq, nbr, Nq, nbr))
    for tau, g in enumerate(g_atoms):
        A = u[:, 3 * tau:3 * tau + 3, :]
        ov += g * np.abs(np.einsum("qxs,pxt->qspt", A.conj(), A)) ** 2
    d = gaussian_delta(w[None, None, :, :] - w[:, :, None, None], wl.sigma_eV, wl.cutoff_sigmas)
    d = d * ok[None, None, :, :]
    raw = np.pi * w ** 2 / (2.0 * HBAR_EVS * Nq) * np.einsum("qspt,qspt->qs", ov, d)
    raw = np.where(ok, raw, 0.0)
    W = np.empty_like(raw)
    for q in range(Nq):
        W[q] = _group_average_matrix(w[q], wl.degen_tol_eV) @ raw[q]
    return W


@dataclasses.dataclass
class BTEResult:
    coeffs: dict
    I: np.ndarray
    J: np.ndarray
    F: np.ndarray
    G: np.ndarray
    W_e: np.ndarray
    W_ph: np.ndarray
    states: np.ndarray          # (nstates, 2): (full k of representative, band)
    outer_iters: int
    inner_iters: list
    residuals: list
    lambdas: list
    converged: bool
    rta_coeffs: dict            # coefficients of the starting responses (the RTA unless init)
    I0: np.ndarray = None
    J0: np.ndarray = None


class _System:
    """Index bookkeeping of the electron states (IBZ representative, active band) and the
    phonon modes (full q mesh, branch), plus the per-entry tables of the rate list."""

    def __init__(self, P: Prepared, R: Rates = None):
        wl = P.wl
        m = wl.model
        self.P, self.R = P, R
        self.nb, self.nbr = m.nb, m.nbranch
        ibzw = ibz_window_points(P) if R is None else R.ibz_win
        st = [(k, b) for k in ibzw for b in range(m.nb) if P.active[k, b]]
        self.states = np.array(st, dtype=np.int64).reshape(-1, 2)
        self.state_of = {tuple(s): i for i, s in enumerate(self.states)}
        if R is not None:
            self.row = np.array([self.state_of[(a, b)] for a, b in zip(R.ik, R.m)], dtype=np.int64)
            self.col = np.array([self.state_of[(P.rep[a], b)] for a, b in zip(R.ikp, R.n)], dtype=np.int64)
            self.Cop = m.sym_cart[P.op[R.ikp]]                    # rotation taking <k'> to k'
            self.mq = minus_q(P, R.iq)
        ks, bs = self.states[:, 0], self.states[:, 1]
        self.eps = P.eps[ks, bs]
        self.v = P.vel[ks, bs]
        self.f = fermi(self.eps, wl.mu_eV, wl.T_K)
        self.ff = self.f * (1.0 - self.f)
        self.inv_stab = 1.0 / P.stab[ks].astype(np.float64)
        if R is not None:
            self.inv_stab_row = self.inv_stab[self.row]
        self.nph = bose(P.w, wl.T_K)
        self.nn1 = self.nph * (1.0 + self.nph)
        self.ph_ok = P.w > wl.omega_min_eV
        V = abs(np.linalg.det(m.lattice)) * ANGSTROM ** 3
        kT = KB_EVK * wl.T_K
        self.Pe = m.spin_deg * E_CHARGE / (V * P.Nk * kT)
        self.Pph = E_CHARGE / (V * P.Nq * kT)
        self.Ycoef = P.Nq / P.Nk          # Y = X^+ N_q / N_k

    # full-BZ sums of state tensors: sum_<k> (1/|stab|) sum_S C_S M C_S^T
    def _bz_tensor(self, weights, vec):
        M = np.einsum("i,ia,ib->ab", weights * self.inv_stab, self.v, vec)
        C = self.P.wl.model.sym_cart
        return np.einsum("sac,cd,sbd->ab", C, M, C)

    def electron_tensors(self, I, J):
        d = self.eps - self.P.wl.mu_eV
        return {
            "sigma": self.Pe * self._bz_tensor(self.ff, J),
            "sigmaS": self.Pe * self._bz_tensor(self.ff, -I),
            "alpha_el": -self.Pe * self._bz_tensor(d * self.ff, J),
            "kappa0_el": -self.Pe * self._bz_tensor(d * self.ff, -I),
        }

    def phonon_tensors(self, F, G):
        P = self.P
        wt = np.where(self.ph_ok, P.w * self.nn1, 0.0)
        return {
            "alpha_ph": self.Pph * np.einsum("qs,qsa,qsb->ab", wt, P.vph, -G),
            "kappa_ph": self.Pph * np.einsum("qs,qsa,qsb->ab", wt, P.vph, F),
        }

    def fold(self, Bt):
        """A(q) = sum_S C_S Bt(S^-1 q): the full-BZ-k sum for phonon q from the IBZ rows."""
        P = self.P
        C = P.wl.model.sym_cart
        out = np.zeros_like(Bt)
        for s_i in range(len(C)):
            src = P.qimages[P.inv_op[s_i]]            # S^-1 q
            if Bt.ndim == 3:
                out += np.einsum("ab,qsb->qsa", C[s_i], Bt[src])
            else:
                out += Bt[src]
        return out


StateSpace = _System


def _residual(new: dict, old: dict, keys) -> float:
    r = 0.0
    for key in keys:
        nrm = np.linalg.norm(new[key])
        if nrm > 0.0:
            r = max(r, np.linalg.norm(new[key] - old[key]) / nrm)
    return r


def coefficients_from_responses(sys_: _System, I, J, F, G) -> dict:
    c = sys_.electron_tensors(I, J)
    c.update(sys_.phonon_tensors(F, G))
    T = sys_.P.wl.T_K
    c["S"] = np.linalg.solve(c["sigma"], c["sigmaS"])
    c["kappa_el"] = c["kappa0_el"] - c["alpha_el"] @ c["S"]
    c["Q_el"] = c["alpha_el"] @ np.linalg.inv(c["sigma"] * T)
    c["Q_ph"] = c["alpha_ph"] @ np.linalg.inv(c["sigma"] * T)
    return c


def solve_coupled_bte(P: Prepared, R: Rates, level: str = "dragged", ko: bool = True, tol: float = None,
                      max_outer: int = 500, max_inner: int = 5000, inner_tol: float = None,
                      init=None) -> BTEResult:
    """RTA (iteration 0), then the unified single-iterator scheme: each phonon iteration
    updates F, G from the current electron responses (drag terms), brings the electron
    equations for both fields to self-consistency against those phonons, and applies
    the Kelvin-Onsager correction.  level: 'rta' | 'dragless' | 'partial' | 'dragged'.
    init: optional starting electron responses (I, J) in place of the RTA ones (I0, J0); the
    phonons start from the RTA either way."""
    wl = P.wl
    tol = wl.tol if tol is None else tol
    inner_tol = 0.1 * tol if inner_tol is None else inner_tol
    sy = _System(P, R)
    T, mu = wl.T_K, wl.mu_eV
    X = R.Xp + R.Xm
    nst = len(sy.states)
    ds = wl.model.spin_deg
    # electron RTA rates (Eq. W^RTA_mk)
    W_e = np.zeros(nst)
    np.add.at(W_e, sy.row, X)
    W_e = W_e / sy.ff
    if getattr(wl, "chimp", None) is not None:   # e-chimp enters the RTA rate only (Matthiessen's rule)
        W_e = W_e + chimp_rates(P, sy.states)
    ok_e = W_e > 0.0
    inv_ffW = np.zeros(nst)
    inv_ffW[ok_e] = 1.0 / (sy.ff[ok_e] * W_e[ok_e])
    # phonon RTA rates (Eq. W^RTA_sq): d_s sum_k Y / (n(1+n)) + background
    Yw = R.Xp * sy.Ycoef * sy.inv_stab_row
    Bt = np.zeros((P.Nq, sy.nbr))
    np.add.at(Bt, (R.iq, R.s), Yw)
    sumY = sy.fold(Bt)
    m = wl.model
    W_bg = m.bg_rate_coeff * (P.w / m.bg_omega_ref_eV) ** 2 * (T / m.bg_T_ref)
    W_ph = np.zeros_like(P.w)
    okp = sy.ph_ok
    W_ph[okp] = ds * sumY[okp] / sy.nn1[okp] + W_bg[okp]
    if getattr(wl, "isotopes", None) is not None:   # ph-isotope enters the RTA rate only
        W_ph[okp] = W_ph[okp] + isotope_rates(P, wl.isotopes)[okp]
    inv_nnW = np.zeros_like(P.w)
    inv_nnW[okp] = 1.0 / (sy.nn1[okp] * W_ph[okp])
    # RTA terms (Eqs. I0/J0, F0/G0)
    I0 = np.zeros((nst, 3))
    J0 = np.zeros((nst, 3))
    I0[ok_e] = ((sy.eps[ok_e] - mu) / T)[:, None] * sy.v[ok_e] / W_e[ok_e, None]
    J0[ok_e] = sy.v[ok_e] / W_e[ok_e, None]
    F0 = np.zeros(P.w.shape + (3,))
    F0[okp] = (P.w[okp] / T)[:, None] * P.vph[okp] / W_ph[okp, None]
    G0 = np.zeros_like(F0)

    def electron_sweep(I, F, drag):
        """I0 + dI^S[I] (+ dI^D[F]) for every state."""
        rotated = np.einsum("eab,eb->ea", sy.Cop, I[sy.col])
        acc = np.zeros_like(I)
        np.add.at(acc, sy.row, rotated * X[:, None])
        if drag:
            d = -F[R.iq, R.s] * R.Xp[:, None] + F[sy.mq, R.s] * R.Xm[:, None]
            np.add.at(acc, sy.row, d)
        return acc * inv_ffW[:, None]

    def phonon_drag(I):
        """dF^D: d_s/(n(1+n) W) sum_{k in FBZ} Y (I_k' - I_k), via the IBZ rows and the fold."""
        rotated = np.einsum("eab,eb->ea", sy.Cop, I[sy.col])
        Bv = np.zeros((P.Nq, sy.nbr, 3))
        np.add.at(Bv, (R.iq, R.s), Yw[:, None] * (rotated - I[sy.row]))
        return ds * sy.fold(Bv) * inv_nnW[..., None]

    I, J, F, G = I0.copy(), J0.copy(), F0.copy(), G0.copy()
    if init is not None:
        I, J = np.array(init[0], dtype=np.float64), np.array(init[1], dtype=np.float64)
    rta = coefficients_from_responses(sy, I, J, F, G)
    res_hist, lam_hist, inner_hist = [], [], []
    ekeys = ("sigma", "sigmaS", "alpha_el", "kappa0_el")
    converged = level == "rta"
    outer = 0

    def inner_loop(I, J, F, G, drag):
        prev = sy.electron_tensors(I, J)
        for it in range(1, max_inner + 1):
            I = I0 + electron_sweep(I, F, drag)
            J = J0 + electron_sweep(J, G, drag)
            cur = sy.electron_tensors(I, J)
            r = _residual(cur, prev, ekeys)
            prev = cur
            if r < inner_tol:
                return I, J, it, True
        return I, J, max_inner, False

    if level == "dragless":
        I, J, n_in, converged = inner_loop(I, J, F, G, drag=False)
        inner_hist.append(n_in)
        outer = 1
    elif level in ("dragged", "partial"):
        prev = rta
        for outer in range(1, max_outer + 1):
            F = F0 + phonon_drag(I)
            G = G0 + phonon_drag(J)
            I, J, n_in, _ = inner_loop(I, J, F, G, drag=True)
            inner_hist.append(n_in)
            if ko:
                # Kelvin-Onsager: I = I_diff + lambda I_drag, I_diff = (eps - mu) J / (e T)
                I_diff = ((sy.eps - mu) / T)[:, None] * J
                I_drag = I - I_diff
                B = sy.electron_tensors(I_drag, J)["sigmaS"]
                A = sy.phonon_tensors(F, G)["alpha_ph"] / T
                nb2 = np.sum(B * B)
                if np.sqrt(nb2) > 1e-30:
                    lam = float(np.sum(A * B) / nb2)
                    I = I_diff + lam * I_drag
                    lam_hist.append(lam)
            cur = coefficients_from_responses(sy, I, J, F, G)
            r = _residual(cur, prev, TENSORS)
            res_hist.append(r)
            prev = cur
            if level == "partial":
                converged = True
                break
            if r < tol:
                converged = True
                break
    coeffs = coefficients_from_responses(sy, I, J, F, G)
    return BTEResult(coeffs=coeffs, I=I, J=J, F=F, G=G, W_e=W_e, W_ph=W_ph, states=sy.states,
                     outer_iters=outer, inner_iters=inner_hist, residuals=res_hist, lambdas=lam_hist,
                     converged=converged, rta_coeffs=rta, I0=I0, J0=J0)
