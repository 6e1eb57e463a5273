"""Seeded synthetic Wannier models and workloads.

This module only BUILDS inputs: tight-binding hoppings H(R_e), mass-scaled force
constants D(R_ph) and Wannier-space couplings g(R_e, R_ph), together with the mesh,
temperature, chemical potential, window and delta-width of each workload.  It holds
none of the method's arithmetic (no Fourier sums, no diagonalisation, no rates, no
BTE); the CUDA path and the oracle both consume the arrays it returns.

The materials of the paper (DFT/EPW silicon, Methods section) are not available;
the models below stand in for them with the same shapes (bands, atoms, branches,
R grids) and value structure (couplings decaying exponentially with |R|).

Conventions shared by both consumers:
  * lattice rows are a1, a2, a3 in Angstrom; R vectors are integer crystal
    coordinates; k and q are reciprocal crystal coordinates (k.R = 2 pi sum k_i R_i).
  * H_R[r, m, n] (eV), complex; H(k) = sum_r exp(i 2 pi k.R_r) H_R[r].
  * D_R[r, a, b] (eV^2), mass-scaled so that the eigenvalues of D(q) are (hbar w)^2.
  * g_R[re, rp, m', n', alpha] (eV), alpha = 3*atom + cartesian.
  * sym_rot[s] integer 3x3 acting on reciprocal crystal coordinates of k,
    sym_cart[s] the same operation acting on Cartesian vectors.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

SEED_BASE = 2109085470


@dataclasses.dataclass
class WannierModel:
    lattice: np.ndarray            # (3,3) Angstrom, rows a1..a3
    mass_amu: np.ndarray           # (nat,)
    tau_cart: np.ndarray           # (nat,3) Angstrom
    nb: int
    Re: np.ndarray                 # (nRe,3) int32
    H_R: np.ndarray                # (nRe,nb,nb) complex128, eV
    Rd: np.ndarray                 # (nRd,3) int32
    D_R: np.ndarray                # (nRd,3nat,3nat) complex128, eV^2
    Rge: np.ndarray                # (nRge,3) int32
    Rgp: np.ndarray                # (nRgp,3) int32
    g_R: np.ndarray                # (nRge,nRgp,nb,nb,3nat) complex128, eV
    omega_ref_eV: float            # hbar*omega at which g_R is quoted
    sym_rot: np.ndarray            # (nsym,3,3) int32
    sym_cart: np.ndarray           # (nsym,3,3) float64
    spin_deg: float = 2.0
    bg_rate_coeff: float = 1.0e12  # 1/s, phonon background rate at omega_ref, T_ref
    bg_omega_ref_eV: float = 0.03
    bg_T_ref: float = 300.0

    @property
    def nat(self) -> int:
        return int(self.mass_amu.shape[0])

    @property
    def nbranch(self) -> int:
        return 3 * self.nat


@dataclasses.dataclass(frozen=True)
class Impurities:
    """Charged dopants of the electron-charged-impurity (e-chimp) channel: one entry per dopant
    species (concentration in cm^-3 and ionization Z), and the zero-frequency dielectric
    constant of the host."""
    n_cm3: tuple
    Z: tuple
    eps_r: float


@dataclasses.dataclass
class Workload:
    name: str
    model: WannierModel
    kmesh: tuple
    qmesh: tuple
    T_K: float
    mu_eV: float
    window: tuple                  # absolute (lo_eV, hi_eV), inclusive
    sigma_eV: float = 0.010
    cutoff_sigmas: float = 8.0
    omega_min_eV: float = 1.0e-4
    degen_tol_eV: float = 1.0e-6
    tol: float = 1.0e-10
    delta: str = "gauss"           # energy-conserving delta: "gauss" (sigma_eV) or "tetra" (no width)
    chimp: Impurities = None       # charged impurities (e-chimp channel), or none
    isotopes: tuple = None         # mass-variance parameter g of each atom (ph-isotope channel), or none


def oh_group() -> np.ndarray:
    """The 48 signed permutation matrices (point group O_h of a cubic lattice)."""
    ops = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            m = np.zeros((3, 3), dtype=np.int32)
            for i in range(3):
                m[i, perm[i]] = signs[i]
            ops.append(m)
    ops.sort(key=lambda m: tuple(m.ravel()))
    # identity first
    ident = [i for i, m in enumerate(ops) if np.array_equal(m, np.eye(3, dtype=np.int32))][0]
    ops.insert(0, ops.pop(ident))
    return np.array(ops, dtype=np.int32)


def identity_group() -> np.ndarray:
    return np.eye(3, dtype=np.int32)[None]


def cube_grid(half: int) -> np.ndarray:
    """Integer vectors with every component in [-half, half], lexicographic order."""
    r = range(-half, half + 1)
    return np.array(list(itertools.product(r, r, r)), dtype=np.int32)


def _index_of(grid: np.ndarray) -> dict:
    return {tuple(v): i for i, v in enumerate(grid)}


def hermitian_pair_symmetrise(g: np.ndarray, Rge: np.ndarray, Rgp: np.ndarray) -> np.ndarray:
    """Impose g_{m'n'a}(Re,Rp) = conj(g_{n'm'a}(-Re, Rp-Re)) (the condition under which
    |g_mn(k,q)| = |g_nm(k+q,-q)|, i.e. the absorption and emission vertices agree).
    Pairs whose partner falls outside the grid are set to zero."""
    ie = _index_of(Rge)
    ip = _index_of(Rgp)
    out = np.zeros_like(g)
    for a, re in enumerate(Rge):
        pe = ie.get(tuple(-re))
        for b, rp in enumerate(Rgp):
            pp = ip.get(tuple(rp - re))
            if pe is None or pp is None:
                continue
            partner = np.conj(np.swapaxes(g[pe, pp], 0, 1))
            out[a, b] = 0.5 * (g[a, b] + partner)
    return out


def hermitian_hoppings(h: np.ndarray, R: np.ndarray) -> np.ndarray:
    """H(-R) = H(R)^dagger, so that H(k) is Hermitian."""
    idx = _index_of(R)
    out = np.empty_like(h)
    for i, r in enumerate(R):
        j = idx[tuple(-r)]
        out[i] = 0.5 * (h[i] + np.conj(h[j].T))
    return out


# --------------------------------------------------------------------------------------
# Model 1: simple cubic, one band, one atom (closed-form bands and phonons)
# --------------------------------------------------------------------------------------

def model_sc1(seed: int = SEED_BASE + 1, a: float = 3.0, t_eV: float = 1.0,
              omega_max_eV: float = 0.030, g0_eV: float = 0.05, noise: float = 0.10) -> WannierModel:
    """Nearest-neighbour tight binding eps = -2t sum cos(k_a a); nearest-neighbour
    springs giving hbar*w_alpha(q) = w_max |sin(q_alpha a/2)| with Cartesian
    eigenvectors; g(Re,Rp) = g0 exp(-(|Re|+|Rp|)/a) (1+xi) on 3^3 x 3^3 R grids, the
    same for the three displacement directions.  xi is drawn once per O_h orbit of
    the pair (Re,Rp) so the model keeps the full cubic symmetry."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lattice = a * np.eye(3)
    nn = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                  dtype=np.int32)
    H_R = np.zeros((7, 1, 1), dtype=np.complex128)
    H_R[1:, 0, 0] = -t_eV
    W2 = omega_max_eV ** 2
    D_R = np.zeros((7, 3, 3), dtype=np.complex128)
    D_R[0] = 0.5 * W2 * np.eye(3)
    for i, r in enumerate(nn[1:], start=1):
        ax = int(np.nonzero(r)[0][0])
        D_R[i, ax, ax] = -0.25 * W2
    grid = cube_grid(1)
    ops = oh_group()
    # noise per orbit of the pair under simultaneous rotation
    keys = {}
    for a_i, re in enumerate(grid):
        for b_i, rp in enumerate(grid):
            key = min((tuple(S @ re), tuple(S @ rp)) for S in ops)
            keys[(a_i, b_i)] = key
    orbit_list = sorted(set(keys.values()))
    xi = dict(zip(orbit_list, rng.uniform(-noise, noise, size=len(orbit_list))))
    g = np.zeros((27, 27, 1, 1, 3), dtype=np.complex128)
    for (a_i, b_i), key in keys.items():
        amp = g0_eV * np.exp(-(np.linalg.norm(grid[a_i]) + np.linalg.norm(grid[b_i]))) * (1.0 + xi[key])
        g[a_i, b_i, 0, 0, :] = amp
    g = hermitian_pair_symmetrise(g, grid, grid)
    return WannierModel(lattice=lattice, mass_amu=np.array([28.0855]), tau_cart=np.zeros((1, 3)), nb=1,
                        Re=nn.copy(), H_R=H_R, Rd=nn.copy(), D_R=D_R, Rge=grid, Rgp=grid.copy(), g_R=g,
                        omega_ref_eV=omega_max_eV, sym_rot=ops, sym_cart=ops.astype(np.float64),
                        bg_omega_ref_eV=omega_max_eV)


# --------------------------------------------------------------------------------------
# Model 3: 8 s-like bands on a simple cubic lattice with the full O_h symmetry
# --------------------------------------------------------------------------------------

def model_sc8(seed: int = SEED_BASE + 3, a: float = 3.0, omega_max_eV: float = 0.060,
              g0_eV: float = 0.01) -> WannierModel:
    """Eight s-like orbitals on one simple-cubic site: four "valence" orbitals with on-site
    energies near -1.2 eV and four "conduction" orbitals near +0.4 eV, hoppings on the
    nearest, edge and corner shells (one real symmetric 8x8 matrix per shell, amplitude
    0.25 eV exp(-|R|/a), the same for every R of a shell, so H(SR) = H(R) for all 48
    operations); the one-atom nearest-neighbour springs of model 1 (w_max 60 meV); real
    couplings g0 exp(-(|Re|+|Rp|)/a) on 3^3 x 3^3 grids, made O_h covariant by the group
    average g^a(Re,Rp) <- (1/48) sum_S sum_b S_ba g^b(S Re, S Rp) and Hermitian-pair
    symmetric.  Real hoppings and couplings keep time-reversal symmetry."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = 8
    lattice = a * np.eye(3)
    grid = cube_grid(1)
    shell = np.abs(grid).sum(axis=1)          # 0 on-site, 1 faces, 2 edges, 3 corners
    onsite = np.concatenate([-1.2 + 0.15 * rng.uniform(-1, 1, 4), 0.4 + 0.15 * rng.uniform(-1, 1, 4)])
    t = np.zeros((4, nb, nb))
    c0 = rng.normal(0.0, 0.05, (nb, nb))
    t[0] = np.diag(onsite) + 0.5 * (c0 + c0.T) - np.diag(np.diag(0.5 * (c0 + c0.T)))
    for sh in (1, 2, 3):
        m = rng.normal(0.0, 1.0, (nb, nb))
        t[sh] = 0.25 * np.exp(-np.sqrt(sh)) * 0.5 * (m + m.T)
    H_R = np.array([t[sh] for sh in shell], dtype=np.complex128)
    # phonons: model 1's nearest-neighbour springs
    nn = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.int32)
    W2 = omega_max_eV ** 2
    D_R = np.zeros((7, 3, 3), dtype=np.complex128)
    D_R[0] = 0.5 * W2 * np.eye(3)
    for i, r in enumerate(nn[1:], start=1):
        ax = int(np.nonzero(r)[0][0])
        D_R[i, ax, ax] = -0.25 * W2
    # couplings: random, decaying, then the O_h group average (covariant in the displacement)
    ops = oh_group()
    idx = _index_of(grid)
    dec = np.exp(-(np.linalg.norm(grid, axis=1)[:, None] + np.linalg.norm(grid, axis=1)[None, :]))
    g = rng.normal(0.0, 1.0, (27, 27, nb, nb, 3)) * (g0_eV * dec)[:, :, None, None, None]
    gs = np.zeros_like(g)
    for S in ops:
        perm = np.array([idx[tuple(S @ r)] for r in grid])   # index of S R
        gs += np.einsum("ba,xymnb->xymna", S.astype(np.float64), g[perm][:, perm])
    gs /= len(ops)
    gs = hermitian_pair_symmetrise(gs.astype(np.complex128), grid, grid)
    return WannierModel(lattice=lattice, mass_amu=np.array([28.0855]), tau_cart=np.zeros((1, 3)), nb=nb,
                        Re=grid.copy(), H_R=H_R, Rd=nn.copy(), D_R=D_R, Rge=grid.copy(), Rgp=grid.copy(), g_R=gs,
                        omega_ref_eV=omega_max_eV, sym_rot=ops, sym_cart=ops.astype(np.float64),
                        bg_omega_ref_eV=omega_max_eV)


# --------------------------------------------------------------------------------------
# Model 2: 4-band seeded random Hamiltonian, 2-atom CsCl-type cubic basis, 6 branches
# --------------------------------------------------------------------------------------

def _cscl_force_constants(K1: float, K2A: float, K2B: float, mA: float, mB: float):
    """Central springs on a CsCl-type lattice (A at 0, B at (1/2,1/2,1/2)a): K1 on the
    8 A-B nearest bonds, K2A / K2B on the 6 A-A / B-B next-nearest bonds.  Returns the
    R list and mass-scaled blocks D(R) (arbitrary energy^2 units, real)."""
    Rd = cube_grid(1)
    idx = _index_of(Rd)
    D = np.zeros((27, 6, 6))
    tau = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    masses = np.array([mA, mB])
    Kmat = {(0, 1): K1, (1, 0): K1, (0, 0): K2A, (1, 1): K2B}
    for i in range(2):
        for j in range(2):
            for R in Rd:
                d = R + tau[j] - tau[i]
                dist = np.linalg.norm(d)
                if dist < 1e-12:
                    continue
                if i != j and abs(dist - np.sqrt(3) / 2) < 1e-9:
                    K = Kmat[(i, j)]
                elif i == j and abs(dist - 1.0) < 1e-9:
                    K = Kmat[(i, j)]
                else:
                    continue
                e = d / dist
                blk = K * np.outer(e, e)
                r = idx[tuple(R)]
                D[r, 3 * i:3 * i + 3, 3 * j:3 * j + 3] -= blk / np.sqrt(masses[i] * masses[j])
                D[idx[(0, 0, 0)], 3 * i:3 * i + 3, 3 * i:3 * i + 3] += blk / masses[i]
    return Rd, D


def model_cscl4(seed: int = SEED_BASE + 2, a: float = 3.0, omega_max_eV: float = 0.060,
                g0_eV: float = 0.01, hop_eV: float = 1.0, nb: int = 4, r_half: int = 2) -> WannierModel:
    """4-band Hamiltonian with seeded normal hoppings 1 eV exp(-|R|/a) on a 5^3 R grid
    (H(-R) = H(R)^dagger, band centre at 0 eV), 2-atom CsCl-type basis (masses 28 and
    16 amu) with seeded nearest / next-nearest central springs scaled so the
    zone-centre optical phonon is omega_max, and normal couplings
    g0 exp(-(|Re|+|Rp|)/a) on 5^3 x 5^3 R grids (stored complex128).

    No point symmetry is kept, but the Wannier functions are taken real (real H(R)
    and g), i.e. the model is time-reversal symmetric as every non-magnetic crystal
    is: eps(-k) = eps(k), v(-k) = -v(k).  Without it the driving terms of the electron
    BTE overlap the collision operator's number-conserving zero mode and the plain
    iteration drifts instead of converging."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lattice = a * np.eye(3)
    R = cube_grid(r_half)
    nR = R.shape[0]
    decay = np.exp(-np.linalg.norm(R, axis=1))
    h = rng.standard_normal((nR, nb, nb)).astype(np.complex128)
    h *= hop_eV * decay[:, None, None]
    H_R = hermitian_hoppings(h, R)
    i0 = _index_of(R)[(0, 0, 0)]
    H_R[i0] -= (np.trace(H_R[i0]).real / nb) * np.eye(nb)
    mA, mB = 28.0855, 15.999
    K = rng.uniform(0.5, 1.5, size=3)
    Rd, D = _cscl_force_constants(K[0], K[1], K[2], mA, mB)
    # zone-centre optical frequency of the central-spring CsCl lattice: (8 K1/3)(1/mA+1/mB)
    w2_opt = (8.0 * K[0] / 3.0) * (1.0 / mA + 1.0 / mB)
    D_R = (D * (omega_max_eV ** 2 / w2_opt)).astype(np.complex128)
    g = rng.standard_normal((nR, nR, nb, nb, 6)).astype(np.complex128)
    g *= g0_eV * (decay[:, None] * decay[None, :])[:, :, None, None, None]
    g = hermitian_pair_symmetrise(g, R, R)
    return WannierModel(lattice=lattice, mass_amu=np.array([mA, mB]),
                        tau_cart=np.array([[0.0, 0.0, 0.0], [0.5 * a, 0.5 * a, 0.5 * a]]), nb=nb,
                        Re=R, H_R=H_R, Rd=Rd, D_R=D_R, Rge=R.copy(), Rgp=R.copy(), g_R=g,
                        omega_ref_eV=omega_max_eV, sym_rot=identity_group(),
                        sym_cart=identity_group().astype(np.float64), bg_omega_ref_eV=omega_max_eV)


# --------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------

def workload_sc1(n: int = 8, nsym_full: bool = True, T_K: float = 300.0) -> Workload:
    """One-band simple-cubic case: 8^3 k and q meshes, mu = +0.3 eV, window mu +- 0.4 eV,
    T = 300 K, Gaussian delta sigma = 10 meV."""
    m = model_sc1()
    if not nsym_full:
        m = dataclasses.replace(m, sym_rot=identity_group(), sym_cart=identity_group().astype(np.float64))
    mu = 0.3
    return Workload(name=f"sc1-{n}^3", model=m, kmesh=(n, n, n), qmesh=(n, n, n), T_K=T_K, mu_eV=mu,
                    window=(mu - 0.4, mu + 0.4), tol=1e-10)


def workload_sc8(n: int = 6, nsym_full: bool = True, T_K: float = 300.0, ratio: int = 1) -> Workload:
    """Eight-band O_h case: n^3 k mesh, (n/ratio)^3 q mesh, mu = 0.2 eV, window mu +- 0.35 eV
    (the lower edge of the conduction group), T = 300 K."""
    m = model_sc8()
    if not nsym_full:
        m = dataclasses.replace(m, sym_rot=identity_group(), sym_cart=identity_group().astype(np.float64))
    mu = 0.2
    q = n // ratio
    return Workload(name=f"sc8-{n}^3", model=m, kmesh=(n, n, n), qmesh=(q, q, q), T_K=T_K, mu_eV=mu,
                    window=(mu - 0.35, mu + 0.35), tol=1e-10)


def workload_cscl4(n: int = 24, T_K: float = 300.0) -> Workload:
    """Four-band, six-branch precision case: n^3 k and q meshes (24^3 at full size),
    mu = 0 eV, window mu +- 0.3 eV, T = 300 K, sigma = 10 meV."""
    m = model_cscl4()
    mu = 0.0
    return Workload(name=f"cscl4-{n}^3", model=m, kmesh=(n, n, n), qmesh=(n, n, n), T_K=T_K, mu_eV=mu,
                    window=(mu - 0.3, mu + 0.3), tol=1e-10)


def instance_grid(n: int, mu0_eV: float = 0.0, half_window_eV: float = 0.25, seed: int = SEED_BASE + 4):
    """n (T_K, mu_eV, window_lo_eV, window_hi_eV) instances: T on a linspace of [100, 500] K and
    mu on a linspace of mu0 +- 0.2 eV, the two paired by a seeded shuffle; each instance's
    window is mu +- half_window, so the active k sets differ from instance to instance."""
    rng = np.random.default_rng(seed)
    T = np.linspace(100.0, 500.0, n)
    mu = mu0_eV + np.linspace(-0.2, 0.2, n)
    rng.shuffle(mu)
    return [(float(t), float(m), float(m - half_window_eV), float(m + half_window_eV)) for t, m in zip(T, mu)]


def model_nbytes(m: WannierModel) -> int:
    return int(sum(x.nbytes for x in (m.lattice, m.mass_amu, m.tau_cart, m.Re, m.H_R, m.Rd, m.D_R,
                                       m.Rge, m.Rgp, m.g_R, m.sym_rot, m.sym_cart)))


# --------------------------------------------------------------------------------------
# Model 4: 8-band O_h semiconductor with a 1.0 eV gap, CsCl-type 2-atom basis, 6 branches
# (the fine-mesh drag case: 7^3 x 7^3 coupling grids, 80^3 k / 40^3 q)
# --------------------------------------------------------------------------------------

def _shell_of(R: np.ndarray) -> np.ndarray:
    """Shell of a vector of the 3^3 grid: 0 on-site, 1 faces, 2 edges, 3 corners."""
    return np.abs(R).sum(axis=-1)


# Dispersion parameters (e, t1, t2, t3) of the two band edges.  With only the face (t1), edge
# (t2) and corner (t3) shells, eps(k) = e + 2 t1 sum_a c_a + 4 t2 sum_{a<b} c_a c_b
# + 8 t3 c_x c_y c_z with c_a = cos(2 pi k_a) is multilinear in (c_x, c_y, c_z), so its extrema
# over the zone sit at the eight corners of the c cube (Gamma, 3 X, 3 M, R).
#   top valence band: t1, t2, t3 > 0, maximum at Gamma: VBM = e + 6 t1 + 12 t2 + 8 t3;
#   lowest conduction band: t1 = -0.8, t2 = 0.3, t3 = 0.05 gives Gamma e-0.8, X e-3.2,
#   M e+0.8, R e+8.0: minimum at the three X points (longitudinal / transverse curvature
#   4 t2 - t1 + 4 t3 ... = 0.4 / 0.8 eV per rad^2, so three anisotropic valleys).
CSCL8_VBM_EV = -0.5
CSCL8_GAP_EV = 1.0
_V0 = (0.35, 0.10, 0.02)
_C0 = (-0.8, 0.3, 0.05)
_C1 = (-0.5, -0.05, -0.01)     # second conduction band: all shells negative, minimum at Gamma
_C1_ABOVE_CBM = 0.12


def cscl8_band_edges():
    """(VBM, CBM) of model_cscl8 in eV, in closed form: the top valence band's maximum at
    Gamma and the lowest conduction band's minimum at X (every even k mesh contains both)."""
    return CSCL8_VBM_EV, CSCL8_VBM_EV + CSCL8_GAP_EV


def _edge_dispersions(rng):
    """On-site energies and shell hoppings (e, t1, t2, t3) of the eight orbitals, valence
    0-3 then conduction 4-7.  Orbitals v0 and c0 carry the band edges (closed form above);
    the others are seeded and placed so that even their extreme values (e +- the summed shell
    magnitudes 6|t1| + 12|t2| + 8|t3|) stay 0.05-0.3 eV below the VBM (valence) or 0.35 eV or
    more above the CBM (c2, c3; c1 is the Gamma valley 0.12 eV above the CBM)."""
    vbm, cbm = cscl8_band_edges()
    par = np.zeros((8, 4))
    span = lambda t: 6 * abs(t[0]) + 12 * abs(t[1]) + 8 * abs(t[2])
    par[0, 1:] = _V0
    par[0, 0] = vbm - (6 * _V0[0] + 12 * _V0[1] + 8 * _V0[2])
    for i in (1, 2, 3):
        t = rng.uniform(-1.0, 1.0, 3) * np.array([0.3, 0.08, 0.02])
        par[i, 1:] = t
        par[i, 0] = vbm - rng.uniform(0.05, 0.3) - span(t)
    par[4, 1:] = _C0
    par[4, 0] = cbm - (2 * _C0[0] * 1 + 4 * _C0[1] * (-1) + 8 * _C0[2] * (-1))
    par[5, 1:] = _C1
    par[5, 0] = cbm + _C1_ABOVE_CBM - (6 * _C1[0] + 12 * _C1[1] + 8 * _C1[2])
    for i in (6, 7):
        t = rng.uniform(-1.0, 1.0, 3) * np.array([0.3, 0.08, 0.02])
        par[i, 1:] = t
        par[i, 0] = cbm + rng.uniform(0.35, 0.8) + span(t)
    return par


def _oh_covariant_couplings(g: np.ndarray, half: int) -> np.ndarray:
    """Group average of couplings g[re][rp][m'][n'][atom][cart] (re, rp flat indices of
    cube_grid(half)) over the 48 operations S of O_h, for the CsCl-type basis (A at the
    origin, B at tau = (1/2,1/2,1/2)):
      g^{kappa a}(Re, Rp) <- (1/48) sum_S sum_b S_ba g^{kappa b}(S Re, S(Rp + tau_kappa) - tau_kappa).
    The B atom's couplings live on the cells whose atom positions Rp + tau lie inside the
    grid's symmetric cube (Rp_i in [-half, half-1]); they are zero elsewhere, and a source cell
    outside that set contributes zero."""
    grid = cube_grid(half)
    idx = _index_of(grid)
    nR = grid.shape[0]
    tau = np.array([0.5, 0.5, 0.5])
    inB = np.all(grid <= half - 1, axis=1)
    out = np.zeros_like(g)
    parts = [np.ascontiguousarray(g[..., kappa, :]) for kappa in (0, 1)]
    for S in oh_group():
        perm = [int(np.nonzero(S[i])[0][0]) for i in range(3)]     # S[i, perm[i]] = sign[i]
        sign = [float(S[i, perm[i]]) for i in range(3)]
        pe = np.array([idx[tuple(S @ r)] for r in grid])
        pB = np.full(nR, -1)
        for i, r in enumerate(grid):
            if inB[i]:
                pB[i] = idx[tuple(np.rint(S.astype(np.float64) @ (r + tau) - tau).astype(np.int32))]
        for kappa, prow in ((0, pe), (1, pB)):
            src = parts[kappa][np.ix_(pe, np.maximum(prow, 0))]
            src[:, prow < 0] = 0.0
            # sum_b S_ba src_b: S_ba is nonzero only for a = perm[b]
            for b in range(3):
                out[..., kappa, perm[b]] += sign[b] * src[..., b]
    return out / 48.0


def _hermitian_pair_cscl(g: np.ndarray, half: int) -> np.ndarray:
    """g_{m'n'}^{kappa a}(Re, Rp) <- (g_{m'n'}(Re, Rp) + conj g_{n'm'}(-Re, Rp - Re)) / 2 for both
    atoms (the same cell shift for A and B); zero where Rp - Re leaves the atom's cells."""
    grid = cube_grid(half)
    idx = _index_of(grid)
    nR = grid.shape[0]
    inB = np.all(grid <= half - 1, axis=1)
    out = np.zeros_like(g)
    for a, re in enumerate(grid):
        pe = idx[tuple(-re)]
        d = grid - re[None, :]
        ok = np.all(np.abs(d) <= half, axis=1)
        pp = np.full(nR, 0)
        pp[ok] = [idx[tuple(v)] for v in d[ok]]
        partner = np.conj(np.swapaxes(g[pe][pp], 1, 2))       # [rp][m'][n'][atom][cart]
        okB = ok & inB & inB[pp]
        out[a, ok, :, :, 0] = 0.5 * (g[a, ok, :, :, 0] + partner[ok, :, :, 0])
        out[a, okB, :, :, 1] = 0.5 * (g[a, okB, :, :, 1] + partner[okB, :, :, 1])
    return out


def model_cscl8(seed: int = SEED_BASE + 5, a: float = 3.0, omega_max_eV: float = 0.060, g0_eV: float = 0.01,
                r_half: int = 3) -> WannierModel:
    """Eight-band O_h semiconductor on a CsCl-type cubic basis (the fine-mesh drag case).

    Electrons: eight s-like orbitals on the A site, four valence and four conduction, with no
    valence-conduction hopping.  Each block is Q diag(h_i(R)) Q^T with a seeded orthogonal Q
    and one hopping per shell (faces, edges, corners) and orbital, so H(SR) = H(R) for the 48
    operations, the eigenvalues are the orbital dispersions and the band edges are closed
    forms (cscl8_band_edges): top valence at Gamma, lowest conduction at the three X points,
    gap exactly 1.0 eV on every even mesh; a second conduction band has its minimum at Gamma
    0.12 eV above the CBM.  Real hoppings (time-reversal symmetric).
    Phonons: model 2's CsCl-type central springs (seeded shell constants, masses 28.0855 /
    15.999 amu, zone-centre optical phonon omega_max), six branches, O_h symmetric.
    Couplings: real normal g0 exp(-(|Re| + |Rp + tau_kappa|)/a) on (2 r_half + 1)^3 x
    (2 r_half + 1)^3 grids (7^3 x 7^3 at full size: 45 M complex values, 723 MB), made O_h
    covariant by the group average and Hermitian-pair symmetric (model_sc8's two steps, with
    the B atom's cell shift under S)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = 8
    lattice = a * np.eye(3)
    Rh = cube_grid(1)
    par = _edge_dispersions(rng)
    Q = []
    for _ in range(2):
        q_, r_ = np.linalg.qr(rng.standard_normal((4, 4)))
        Q.append(q_ * np.sign(np.diag(r_))[None, :])
    sh = _shell_of(Rh)
    H_R = np.zeros((Rh.shape[0], nb, nb), dtype=np.complex128)
    for r in range(Rh.shape[0]):
        h = par[:, 0] if sh[r] == 0 else par[:, sh[r]]
        H_R[r, :4, :4] = Q[0] @ np.diag(h[:4]) @ Q[0].T
        H_R[r, 4:, 4:] = Q[1] @ np.diag(h[4:]) @ Q[1].T
    mA, mB = 28.0855, 15.999
    K = rng.uniform(0.5, 1.5, size=3)
    Rd, D = _cscl_force_constants(K[0], K[1], K[2], mA, mB)
    w2_opt = (8.0 * K[0] / 3.0) * (1.0 / mA + 1.0 / mB)
    D_R = (D * (omega_max_eV ** 2 / w2_opt)).astype(np.complex128)
    # couplings g[re][rp][m'][n'][atom][cart], decaying with |Re| and the displaced atom's |Rp + tau|
    grid = cube_grid(r_half)
    rre = np.linalg.norm(grid, axis=1)
    rpB = np.linalg.norm(grid + 0.5, axis=1)
    g = rng.standard_normal((grid.shape[0], grid.shape[0], nb, nb, 2, 3))
    g[..., 0, :] *= g0_eV * np.exp(-(rre[:, None] + rre[None, :]))[:, :, None, None, None]
    g[..., 1, :] *= g0_eV * np.exp(-(rre[:, None] + rpB[None, :]))[:, :, None, None, None]
    g = _oh_covariant_couplings(g, r_half)
    g = _hermitian_pair_cscl(g.astype(np.complex128), r_half)
    g_R = np.ascontiguousarray(g.reshape(grid.shape[0], grid.shape[0], nb, nb, 6))
    ops = oh_group()
    return WannierModel(lattice=lattice, mass_amu=np.array([mA, mB]),
                        tau_cart=np.array([[0.0, 0.0, 0.0], [0.5 * a, 0.5 * a, 0.5 * a]]), nb=nb,
                        Re=Rh, H_R=H_R, Rd=Rd, D_R=D_R, Rge=grid, Rgp=grid.copy(), g_R=g_R,
                        omega_ref_eV=omega_max_eV, sym_rot=ops, sym_cart=ops.astype(np.float64),
                        bg_omega_ref_eV=omega_max_eV)


def workload_cscl8(n_k: int = 80, n_q: int = 40, r_half: int = 3, nsym_full: bool = True, T_K: float = 300.0,
                   model: WannierModel = None, above_cbm_eV: float = 0.25) -> Workload:
    """Fine-mesh drag case: n_k^3 k mesh (irreducible wedge under O_h), n_q^3 q mesh,
    mu = E_CBM - 0.1 eV, T = 300 K; the transport window holds the conduction states up to
    0.25 eV (above_cbm_eV) above the CBM: (E_CBM - gap/2, E_CBM + 0.25 eV), the lower edge at
    mid-gap so no state lies near it."""
    m = model_cscl8(r_half=r_half) if model is None else model
    if not nsym_full:
        m = dataclasses.replace(m, sym_rot=identity_group(), sym_cart=identity_group().astype(np.float64))
    _, cbm = cscl8_band_edges()
    return Workload(name=f"cscl8-{n_k}^3/{n_q}^3", model=m, kmesh=(n_k,) * 3, qmesh=(n_q,) * 3, T_K=T_K,
                    mu_eV=cbm - 0.1, window=(cbm - 0.5 * CSCL8_GAP_EV, cbm + above_cbm_eV), tol=1e-10)
