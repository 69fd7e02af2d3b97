"""Seeded synthetic molecule-shaped quadrature grids, densities and trial densities.

This module produces the *inputs* of the VV10 double grid sum.  It stands in for what a
quantum-chemistry code hands the nonlocal kernel: an atom-centred quadrature grid
(Sec. II.A: Becke-style atom-centred quadrature, points r_i and weights w_i), the
ground-state density rho_i and its gradient on that grid (Eq. for omega/kappa need
rho and gamma = |grad rho|^2), and the trial densities (rho^t_i, grad rho^t_i) of the
contracted orbital Hessian (Eq. frhot and the definition of rho^t, gamma^t that follows
it).  The paper's own data sets and Q-Chem grids are not available; every molecule,
grid and density here is synthetic and seeded.

It contains none of the VV10 arithmetic (no omega, kappa, Phi or pair sum): both the
CUDA path and the CPU oracle consume its arrays, and neither imports the other.

Recipe (all lengths in bohr, FP64):
* radial grid: Euler-Maclaurin with the Murray-Handy-Laming map,
  r_k = R_A k^2/(n+1-k)^2, w_k = 2 R_A^3 (n+1) k^5/(n+1-k)^7 (r^2 dr included);
* angular grid: Fibonacci sphere, z_m = 1-(2m+1)/n, phi_m = m*pi*(3-sqrt 5), w = 4 pi/n;
* Becke fuzzy-cell partition (three smoothing iterations, no size adjustment) evaluated
  over the owning atom plus its 8 nearest other atoms (exact Becke for <= 9 atoms);
  weights are then fixed inputs;
* density: per atom three normalised s-Gaussians, exponents 0.3, sqrt(0.3*20), 20,
  each holding Z/3 electrons; analytic gradient;
* trial densities: analytic nuclear-displacement derivatives d rho/d R_{A,c}
  and their spatial gradients, P = 3 N_atom, ordered t = 3A + c;
* weight directions: analytic nuclear derivatives of the weights w^B = d w / d R_B
  (Becke partition differentiated with the points moving with their atoms), 3 N_atom
  directions ordered t = 3B + c.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

BOHR_PER_ANGSTROM = 1.8897261246
Z_OF = {"H": 1, "C": 6, "N": 7, "O": 8}
# Radial scale R_A of the Murray-Handy-Laming map (bohr); a free choice of this recipe.
RADIAL_SCALE = {"H": 1.0, "C": 1.5, "N": 1.4, "O": 1.3}
GAUSS_EXPONENTS = (0.3, math.sqrt(0.3 * 20.0), 20.0)
BECKE_NEIGHBOURS = 8


@dataclasses.dataclass
class Molecule:
    symbols: List[str]
    coords: np.ndarray  # (n_atom, 3) bohr

    @property
    def n_atom(self) -> int:
        return len(self.symbols)

    @property
    def charges(self) -> np.ndarray:
        return np.array([Z_OF[s] for s in self.symbols], dtype=np.float64)


@dataclasses.dataclass
class GridDensity:
    """Grid points with the density on them (all FP64, C-contiguous)."""

    coords: np.ndarray         # (N, 3)
    weights: np.ndarray        # (N,)
    rho: np.ndarray            # (N,)
    grad_rho: np.ndarray       # (N, 3)
    atom_of_point: np.ndarray  # (N,) int32, points are contiguous per atom
    molecule: Molecule

    @property
    def n(self) -> int:
        return int(self.weights.shape[0])


# ----------------------------------------------------------------------------- molecules

def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random SO(3) matrix from a normalised Gaussian quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def water() -> Molecule:
    """O at the origin, two H at 0.96 A with a 104.5 degree angle, in the xy plane."""
    d = 0.96 * BOHR_PER_ANGSTROM
    half = math.radians(104.5) / 2
    coords = np.array([[0.0, 0.0, 0.0],
                       [d * math.sin(half), d * math.cos(half), 0.0],
                       [-d * math.sin(half), d * math.cos(half), 0.0]])
    return Molecule(["O", "H", "H"], coords)


def water_cluster(rng: np.random.Generator, n_water: int = 6) -> Molecule:
    """Rigid waters with O on a puckered ring, neighbouring O-O = 2.8 +- 0.2 A.

    Each water is rotated by a uniform random rotation about its O; a rotation is
    redrawn while any intermolecular H-H or O-H distance is below 1.5 A.
    """
    w = water()
    # Ring radius giving a 2.8 A side for a regular n-gon, perturbed per vertex.
    side = 2.8 * BOHR_PER_ANGSTROM
    radius = side / (2 * math.sin(math.pi / n_water))
    o_pos = []
    for k in range(n_water):
        r = radius + rng.uniform(-0.2, 0.2) * BOHR_PER_ANGSTROM
        ang = 2 * math.pi * k / n_water
        z = (0.25 if k % 2 == 0 else -0.25) * BOHR_PER_ANGSTROM
        o_pos.append(np.array([r * math.cos(ang), r * math.sin(ang), z]))
    symbols: List[str] = []
    coords: List[np.ndarray] = []
    min_d = 1.5 * BOHR_PER_ANGSTROM
    for k in range(n_water):
        for _ in range(1000):
            rot = _random_rotation(rng)
            cand = (w.coords @ rot.T) + o_pos[k]
            ok = True
            for s_new, c_new in zip(w.symbols, cand):
                for s_old, c_old in zip(symbols, coords):
                    if s_new == "O" and s_old == "O":
                        continue
                    if np.linalg.norm(c_new - c_old) < min_d:
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                break
        symbols.extend(w.symbols)
        coords.extend(list(cand))
    return Molecule(symbols, np.array(coords))


def random_chon(rng: np.random.Generator, n_atom: int) -> Molecule:
    """Random tree-grown C/H/N/O molecule (element odds 0.4/0.4/0.1/0.1).

    Each new atom is bonded to a random existing atom at U(1.0, 1.5) A in a random
    direction; a placement closer than 1.0 A to any other atom is redrawn.
    """
    elems = ["C", "H", "N", "O"]
    probs = [0.4, 0.4, 0.1, 0.1]
    symbols = [str(rng.choice(elems, p=probs))]
    coords = [np.zeros(3)]
    lo, hi, dmin = (x * BOHR_PER_ANGSTROM for x in (1.0, 1.5, 1.0))
    while len(symbols) < n_atom:
        parent = coords[int(rng.integers(len(coords)))]
        cand = parent + rng.uniform(lo, hi) * _random_unit(rng)
        if min(np.linalg.norm(cand - c) for c in coords) < dmin * 0.999:
            continue
        symbols.append(str(rng.choice(elems, p=probs)))
        coords.append(cand)
    c = np.array(coords)
    return Molecule(symbols, c - c.mean(axis=0))


def fragment_cluster(rng: np.random.Generator, n_frag: int = 4, frag_atoms: int = 6) -> Molecule:
    """n_frag random CHON fragments whose closest inter-fragment atoms are 3-4 A apart."""
    frags = [random_chon(rng, frag_atoms) for _ in range(n_frag)]
    symbols = list(frags[0].symbols)
    coords = frags[0].coords.copy()
    for f in frags[1:]:
        target = rng.uniform(3.0, 4.0) * BOHR_PER_ANGSTROM
        direction = _random_unit(rng)
        rot = _random_rotation(rng)
        fc = f.coords @ rot.T

        def gap(t: float) -> float:
            moved = fc + t * direction
            d = np.linalg.norm(moved[:, None, :] - coords[None, :, :], axis=-1)
            return float(d.min())

        t_lo, t_hi = 0.0, 10.0
        while gap(t_hi) < target:
            t_hi *= 2
        for _ in range(60):  # bisection on the translation length
            mid = 0.5 * (t_lo + t_hi)
            if gap(mid) < target:
                t_lo = mid
            else:
                t_hi = mid
        symbols.extend(f.symbols)
        coords = np.vstack([coords, fc + t_hi * direction])
    return Molecule(symbols, coords - coords.mean(axis=0))


# ----------------------------------------------------------------------------- grids

def radial_grid(n: int, scale: float):
    k = np.arange(1, n + 1, dtype=np.float64)
    r = scale * k ** 2 / (n + 1 - k) ** 2
    w = 2.0 * scale ** 3 * (n + 1) * k ** 5 / (n + 1 - k) ** 7
    return r, w


def fibonacci_sphere(n: int):
    m = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * m + 1.0) / n
    phi = m * math.pi * (3.0 - math.sqrt(5.0))
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    u = np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)
    return u, np.full(n, 4.0 * math.pi / n)


def _becke_s(mu: np.ndarray) -> np.ndarray:
    p = mu
    for _ in range(3):
        p = 1.5 * p - 0.5 * p ** 3
    return 0.5 * (1.0 - p)


def _becke_fraction(points: np.ndarray, owner: int, atoms: np.ndarray) -> np.ndarray:
    """Becke cell weight of atom `owner` at each point, over owner + nearest others."""
    n_atom = atoms.shape[0]
    d = np.linalg.norm(points[:, None, :] - atoms[None, :, :], axis=-1)  # (n, n_atom)
    if n_atom == 1:
        return np.ones(points.shape[0])
    k = min(BECKE_NEIGHBOURS, n_atom - 1)
    d_other = d.copy()
    d_other[:, owner] = np.inf
    nbr = np.argpartition(d_other, k - 1, axis=1)[:, :k]                # (n, k)
    idx = np.concatenate([np.full((points.shape[0], 1), owner), nbr], axis=1)  # (n, m)
    dm = np.take_along_axis(d, idx, axis=1)                              # (n, m)
    r_atoms = np.linalg.norm(atoms[:, None, :] - atoms[None, :, :], axis=-1)
    rab = r_atoms[idx[:, :, None], idx[:, None, :]]                      # (n, m, m)
    m = idx.shape[1]
    eye = np.eye(m, dtype=bool)[None]
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = (dm[:, :, None] - dm[:, None, :]) / rab
    s = np.where(eye, 1.0, _becke_s(np.clip(np.nan_to_num(mu), -1.0, 1.0)))
    cell = np.prod(s, axis=2)                                            # (n, m)
    return cell[:, 0] / cell.sum(axis=1)


def molecular_grid(mol: Molecule, n_rad: int, n_ang: int, chunk: int = 100_000):
    """Atom-centred grid: (coords (N,3), weights (N,), atom_of_point (N,) int32)."""
    u, wa = fibonacci_sphere(n_ang)
    pts, wts, own = [], [], []
    for a, (sym, centre) in enumerate(zip(mol.symbols, mol.coords)):
        r, wr = radial_grid(n_rad, RADIAL_SCALE[sym])
        p = (r[:, None, None] * u[None, :, :]).reshape(-1, 3) + centre
        w = (wr[:, None] * wa[None, :]).reshape(-1)
        frac = np.empty(p.shape[0])
        for s0 in range(0, p.shape[0], chunk):
            frac[s0:s0 + chunk] = _becke_fraction(p[s0:s0 + chunk], a, mol.coords)
        pts.append(p)
        wts.append(w * frac)
        own.append(np.full(p.shape[0], a, dtype=np.int32))
    return np.concatenate(pts), np.concatenate(wts), np.concatenate(own)


def _becke_s_ds(mu: np.ndarray):
    """Becke's cutoff s(mu) and ds/dmu (three iterations of p -> 1.5 p - 0.5 p^3)."""
    p, dp = mu, np.ones_like(mu)
    for _ in range(3):
        dp = (1.5 - 1.5 * p * p) * dp
        p = 1.5 * p - 0.5 * p ** 3
    return 0.5 * (1.0 - p), -0.5 * dp


def _becke_fraction_grad(points: np.ndarray, owner: int, atoms: np.ndarray):
    """The Becke cell weight of atom `owner` at each point (as _becke_fraction) and its
    derivative with respect to every atom position, the points moving with their owner:
    (frac (n,), grad (n, n_atom, 3)).  Atoms outside a point's neighbour set contribute
    nothing; the owner's derivative follows from translational invariance."""
    n_atom, n = atoms.shape[0], points.shape[0]
    grad = np.zeros((n, n_atom, 3))
    if n_atom == 1:
        return np.ones(n), grad
    d = np.linalg.norm(points[:, None, :] - atoms[None, :, :], axis=-1)
    k = min(BECKE_NEIGHBOURS, n_atom - 1)
    d_other = d.copy()
    d_other[:, owner] = np.inf
    nbr = np.argpartition(d_other, k - 1, axis=1)[:, :k]
    idx = np.concatenate([np.full((n, 1), owner), nbr], axis=1)          # (n, m)
    m = idx.shape[1]
    ra = atoms[idx]                                                      # (n, m, 3)
    dvec = points[:, None, :] - ra
    dm = np.linalg.norm(dvec, axis=-1)                                   # (n, m)
    u = dvec / dm[..., None]
    Rv = ra[:, :, None, :] - ra[:, None, :, :]                           # (n, m, m, 3)
    rab = np.linalg.norm(Rv, axis=-1)
    eye = np.eye(m, dtype=bool)[None]
    safe = np.where(eye, 1.0, rab)
    mu = np.clip(np.where(eye, 0.0, (dm[:, :, None] - dm[:, None, :]) / safe), -1.0, 1.0)
    e = Rv / safe[..., None]
    sv, ds = _becke_s_ds(mu)
    sv = np.where(eye, 1.0, sv)
    ds = np.where(eye, 0.0, ds)
    cell = np.prod(sv, axis=2)                                           # (n, m)
    # product over E != D of s_CE, from prefix and suffix products along E
    pre = np.ones_like(sv)
    pre[:, :, 1:] = np.cumprod(sv[:, :, :-1], axis=2)
    suf = np.ones_like(sv)
    suf[:, :, :-1] = np.cumprod(sv[:, :, ::-1], axis=2)[:, :, ::-1][:, :, 1:]
    G = ds * pre * suf                                                   # (n, C, D)
    # d mu_CD / d R_C = -(u_C + mu_CD e_CD)/R_CD,  d mu_CD / d R_D = (u_D + mu_CD e_CD)/R_CD
    dC = np.where(eye[..., None], 0.0, -(u[:, :, None, :] + mu[..., None] * e) / safe[..., None])
    dD = np.where(eye[..., None], 0.0, (u[:, None, :, :] + mu[..., None] * e) / safe[..., None])
    dcell = G[..., None] * dD                                            # (n, C, X, 3), X != C
    ar = np.arange(m)
    dcell[:, ar, ar, :] += np.einsum("ncd,ncdk->nck", G, dC)             # X = C
    Z = cell.sum(axis=1)
    dZ = dcell.sum(axis=1)                                               # (n, X, 3)
    frac = cell[:, 0] / Z
    dP = (dcell[:, 0] * Z[:, None, None] - cell[:, 0][:, None, None] * dZ) / (Z * Z)[:, None, None]
    dP[:, 0] = -dP[:, 1:].sum(axis=1)
    grad[np.arange(n)[:, None], idx] = dP
    return frac, grad


def weight_directions(mol: Molecule, n_rad: int, n_ang: int, chunk: int = 20_000) -> np.ndarray:
    """Nuclear derivatives of the quadrature weights of molecular_grid(mol, n_rad, n_ang):
    w^B_j = d w_j / d R_{B,c} with every point moving with its atom (the w^A, w^B of
    Sec. II), as 3 N_atom directions ordered t = 3 B + c: array (3 N_atom, N)."""
    u, wa = fibonacci_sphere(n_ang)
    out = []
    for a, (sym, centre) in enumerate(zip(mol.symbols, mol.coords)):
        r, wr = radial_grid(n_rad, RADIAL_SCALE[sym])
        p = (r[:, None, None] * u[None, :, :]).reshape(-1, 3) + centre
        base = (wr[:, None] * wa[None, :]).reshape(-1)
        gw = np.empty((p.shape[0], mol.n_atom, 3))
        for s0 in range(0, p.shape[0], chunk):
            _, gw[s0:s0 + chunk] = _becke_fraction_grad(p[s0:s0 + chunk], a, mol.coords)
        out.append(base[:, None, None] * gw)
    return np.ascontiguousarray(np.concatenate(out).reshape(-1, 3 * mol.n_atom).T)


# ----------------------------------------------------------------------------- densities

def _gauss_coeffs(z: float) -> np.ndarray:
    a = np.array(GAUSS_EXPONENTS)
    return (z / 3.0) * (a / math.pi) ** 1.5


def density(mol: Molecule, points: np.ndarray):
    """rho (N,) and grad rho (N,3) of the sum of atomic s-Gaussians."""
    rho = np.zeros(points.shape[0])
    grad = np.zeros_like(points)
    alphas = np.array(GAUSS_EXPONENTS)
    for z, centre in zip(mol.charges, mol.coords):
        d = points - centre
        r2 = np.einsum("ij,ij->i", d, d)
        for c, a in zip(_gauss_coeffs(z), alphas):
            e = c * np.exp(-a * r2)
            rho += e
            grad += (-2.0 * a * e)[:, None] * d
    return rho, grad


def trial_densities(mol: Molecule, points: np.ndarray, atoms: Optional[Sequence[int]] = None,
                    dtype=np.float64):
    """Nuclear-displacement trial densities.

    rho^{A,c}(r) = d rho / d R_{A,c} = sum_k c_k 2 a_k (r_c - R_{A,c}) exp(-a_k |r-R_A|^2),
    d_d rho^{A,c} = sum_k c_k 2 a_k exp(...) [delta_cd - 2 a_k (r_c-R_{A,c})(r_d-R_{A,d})].
    Returns rho_t (P, N) and grad_rho_t (P, N, 3) with t = 3*A + c.
    """
    atoms = list(range(mol.n_atom)) if atoms is None else list(atoms)
    n = points.shape[0]
    P = 3 * len(atoms)
    rho_t = np.zeros((P, n), dtype=dtype)
    grad_t = np.zeros((P, n, 3), dtype=dtype)
    alphas = np.array(GAUSS_EXPONENTS)
    eye = np.eye(3)
    for ia, a_idx in enumerate(atoms):
        z, centre = mol.charges[a_idx], mol.coords[a_idx]
        d = points - centre
        r2 = np.einsum("ij,ij->i", d, d)
        rt = np.zeros((n, 3))
        gt = np.zeros((n, 3, 3))
        for c, a in zip(_gauss_coeffs(z), alphas):
            e = 2.0 * a * c * np.exp(-a * r2)
            rt += e[:, None] * d
            gt += e[:, None, None] * (eye[None] - 2.0 * a * d[:, :, None] * d[:, None, :])
        for cc in range(3):
            rho_t[3 * ia + cc] = rt[:, cc]
            grad_t[3 * ia + cc] = gt[:, cc, :]
    return rho_t, grad_t


def density_hessian(mol: Molecule, points: np.ndarray) -> np.ndarray:
    """The spatial Hessian of rho (N, 3, 3) for the sum of atomic s-Gaussians."""
    H = np.zeros((points.shape[0], 3, 3))
    alphas = np.array(GAUSS_EXPONENTS)
    eye = np.eye(3)
    for z, centre in zip(mol.charges, mol.coords):
        d = points - centre
        r2 = np.einsum("ij,ij->i", d, d)
        for c, a in zip(_gauss_coeffs(z), alphas):
            e = c * np.exp(-a * r2)
            H += e[:, None, None] * (4.0 * a * a * d[:, :, None] * d[:, None, :] - 2.0 * a * eye[None])
    return H


def nuclear_density_derivatives(mol: Molecule, points: np.ndarray, atom_of_point: np.ndarray):
    """d rho_i / d R_{A,c} and d grad rho_i / d R_{A,c} at grid points that move with their atom
    (r_i - R_owner fixed): the derivative at a fixed point (trial_densities) plus, for the
    owner atom, the spatial derivative at the point.  (3 N_atom, N) and (3 N_atom, N, 3),
    t = 3 A + c."""
    rt, gt = trial_densities(mol, points)
    _, grad = density(mol, points)
    H = density_hessian(mol, points)
    for A in range(mol.n_atom):
        m = atom_of_point == A
        for c in range(3):
            rt[3 * A + c, m] += grad[m, c]
            gt[3 * A + c, m] += H[m, c, :]
    return rt, gt


def nuclear_density_second_derivatives(mol: Molecule, points: np.ndarray,
                                       atom_of_point: np.ndarray):
    """d^2 rho_i / dR_a dR_b and d^2 grad rho_i / dR_a dR_b (a = 3 A + c) at grid points that move
    with their atom.  With x_C = r_i - R_C and f_A(i) = [A owns i] - [A = C], each atomic
    density rho_C contributes f_A f_B d^2 rho_C / dx_c dx_d (and the third derivatives for the
    gradient).  (3 N_atom, 3 N_atom, N) and (3 N_atom, 3 N_atom, N, 3)."""
    n, na = points.shape[0], mol.n_atom
    P = 3 * na
    r2d = np.zeros((P, P, n))
    g2d = np.zeros((P, P, n, 3))
    alphas = np.array(GAUSS_EXPONENTS)
    eye = np.eye(3)
    for C, (z, cen) in enumerate(zip(mol.charges, mol.coords)):
        x = points - cen
        xx = np.einsum("ij,ij->i", x, x)
        H = np.zeros((n, 3, 3))
        T = np.zeros((n, 3, 3, 3))  # T[e, c, d] = d^3 rho_C / dx_e dx_c dx_d
        for c, a in zip(_gauss_coeffs(z), alphas):
            e = c * np.exp(-a * xx)
            H += e[:, None, None] * (4 * a * a * x[:, :, None] * x[:, None, :] - 2 * a * eye[None])
            T += e[:, None, None, None] * (
                -8 * a ** 3 * x[:, :, None, None] * x[:, None, :, None] * x[:, None, None, :]
                + 4 * a * a * (eye[None, :, :, None] * x[:, None, None, :]
                               + eye[None, :, None, :] * x[:, None, :, None]
                               + eye[None, None, :, :] * x[:, :, None, None]))
        f = np.stack([(atom_of_point == A).astype(float) - (1.0 if A == C else 0.0)
                      for A in range(na)])                                  # (na, n)
        ff = f[:, None, :] * f[None, :, :]                                  # (na, na, n)
        r2d += np.einsum("abn,ncd->acbdn", ff, H).reshape(P, P, n)
        g2d += np.einsum("abn,necd->acbdne", ff, T).reshape(P, P, n, 3)
    return r2d, g2d


def weight_second_derivatives(mol: Molecule, n_rad: int, n_ang: int, h: float = 1e-5) -> np.ndarray:
    """d^2 w_i / dR_a dR_b (3 N_atom, 3 N_atom, N): central differences (step h bohr) of the
    analytic first derivatives of weight_directions."""
    P = 3 * mol.n_atom
    out = None
    for b in range(P):
        Ws = []
        for sg in (1.0, -1.0):
            c = mol.coords.copy()
            c[b // 3, b % 3] += sg * h
            Ws.append(weight_directions(Molecule(mol.symbols, c), n_rad, n_ang))
        if out is None:
            out = np.zeros((P, P, Ws[0].shape[1]))
        out[:, b] = (Ws[0] - Ws[1]) / (2 * h)
    return out


def trial_densities_torch(mol: Molecule, points, atoms: Optional[Sequence[int]] = None,
                          out_rho=None, out_grad=None):
    """trial_densities evaluated with torch on the device of `points` (an (N, 3) float64
    tensor), for inputs too large to build on the host.  Writes into out_rho (P, N) and
    out_grad (P, N, 3) when given (any float64 views), else allocates them."""
    import torch
    atoms = list(range(mol.n_atom)) if atoms is None else list(atoms)
    n = points.shape[0]
    P = 3 * len(atoms)
    kw = dict(dtype=torch.float64, device=points.device)
    rho_t = torch.empty(P, n, **kw) if out_rho is None else out_rho
    grad_t = torch.empty(P, n, 3, **kw) if out_grad is None else out_grad
    eye = torch.eye(3, **kw)
    for ia, a_idx in enumerate(atoms):
        z = float(mol.charges[a_idx])
        d = points - torch.as_tensor(mol.coords[a_idx], **kw)
        r2 = (d * d).sum(dim=1)
        rt = torch.zeros(n, 3, **kw)
        gt = torch.zeros(n, 3, 3, **kw)
        for c, a in zip(_gauss_coeffs(z), GAUSS_EXPONENTS):
            e = 2.0 * a * float(c) * torch.exp(-a * r2)
            rt += e[:, None] * d
            gt += e[:, None, None] * (eye[None] - 2.0 * a * d[:, :, None] * d[:, None, :])
        rho_t[3 * ia:3 * ia + 3] = rt.T
        grad_t[3 * ia:3 * ia + 3] = gt.permute(1, 0, 2)
    return rho_t, grad_t


# ----------------------------------------------------------------------------- configs

def make_system(mol: Molecule, n_rad: int, n_ang: int) -> GridDensity:
    coords, weights, own = molecular_grid(mol, n_rad, n_ang)
    rho, grad = density(mol, coords)
    return GridDensity(np.ascontiguousarray(coords), np.ascontiguousarray(weights),
                       np.ascontiguousarray(rho), np.ascontiguousarray(grad),
                       np.ascontiguousarray(own), mol)


SEED_BASE = 20220830


# ----------------------------------------------------------------------------- AO basis

# Uncontracted Cartesian Gaussian shells per element, (l, exponent in bohr^-2), l = 0 (s) or 1 (p):
# a free choice of this recipe, loosely double-zeta-like.
AO_SHELLS = {
    "H": [(0, 1.3), (0, 0.25)],
    "C": [(0, 6.0), (0, 1.0), (0, 0.25), (1, 1.2), (1, 0.3)],
    "N": [(0, 7.5), (0, 1.3), (0, 0.3), (1, 1.5), (1, 0.35)],
    "O": [(0, 9.0), (0, 1.6), (0, 0.35), (1, 1.8), (1, 0.4)],
}


@dataclasses.dataclass
class AOBasis:
    """Basis functions phi_mu = N r_c^l exp(-alpha |r - A|^2) (c = the Cartesian component of
    a p function), each normalised to unit self-overlap."""

    centers: np.ndarray  # (nbf, 3)
    alpha: np.ndarray    # (nbf,)
    comp: np.ndarray     # (nbf,) int: -1 for s, 0/1/2 for p_x/p_y/p_z
    atom: np.ndarray     # (nbf,) int
    norm: np.ndarray     # (nbf,)

    @property
    def nbf(self) -> int:
        return int(self.alpha.shape[0])


def ao_basis(mol: Molecule) -> AOBasis:
    cen, al, cp, at = [], [], [], []
    for a, (sym, c) in enumerate(zip(mol.symbols, mol.coords)):
        for l, e in AO_SHELLS[sym]:
            for k in ([-1] if l == 0 else [0, 1, 2]):
                cen.append(c)
                al.append(e)
                cp.append(k)
                at.append(a)
    al = np.array(al)
    cp = np.array(cp, dtype=np.int64)
    # unit self-overlap: s: (2 alpha/pi)^(3/4); p: (2 alpha/pi)^(3/4) * 2 sqrt(alpha)
    norm = (2.0 * al / math.pi) ** 0.75 * np.where(cp >= 0, 2.0 * np.sqrt(al), 1.0)
    return AOBasis(np.array(cen), al, cp, np.array(at, dtype=np.int64), norm)


def ao_values(basis: AOBasis, points: np.ndarray):
    """(phi (n, nbf), grad phi (n, nbf, 3)) at the points."""
    d = points[:, None, :] - basis.centers[None, :, :]          # (n, nbf, 3)
    r2 = np.einsum("nmk,nmk->nm", d, d)
    g = basis.norm[None, :] * np.exp(-basis.alpha[None, :] * r2)  # radial part
    is_p = basis.comp >= 0
    cidx = np.where(is_p, basis.comp, 0)
    dc = np.take_along_axis(d, cidx[None, :, None].repeat(d.shape[0], 0), axis=2)[..., 0]
    ang = np.where(is_p[None, :], dc, 1.0)
    phi = ang * g
    dphi = -2.0 * basis.alpha[None, :, None] * d * phi[..., None]
    # p functions: + N exp(-alpha r^2) along their own component
    eye = np.zeros((basis.nbf, 3))
    eye[np.arange(basis.nbf)[is_p], basis.comp[is_p]] = 1.0
    dphi += g[..., None] * eye[None, :, :]
    return np.ascontiguousarray(phi), np.ascontiguousarray(dphi)


def ao_second_derivatives(basis: AOBasis, points: np.ndarray) -> np.ndarray:
    """The Hessians of the basis functions at the points, (n, nbf, 3, 3).  With d = r - A and
    g = N exp(-alpha |d|^2): s functions (phi = g) d^2 phi = (4 alpha^2 d d^T - 2 alpha I) phi;
    p functions (phi = d_c g) add -2 alpha g (e_c d^T + d e_c^T)."""
    d = points[:, None, :] - basis.centers[None, :, :]          # (n, nbf, 3)
    r2 = np.einsum("nmk,nmk->nm", d, d)
    g = basis.norm[None, :] * np.exp(-basis.alpha[None, :] * r2)
    is_p = basis.comp >= 0
    cidx = np.where(is_p, basis.comp, 0)
    dc = np.take_along_axis(d, cidx[None, :, None].repeat(d.shape[0], 0), axis=2)[..., 0]
    phi = np.where(is_p[None, :], dc, 1.0) * g
    al = basis.alpha[None, :, None, None]
    H = (4.0 * al ** 2 * d[..., :, None] * d[..., None, :]
         - 2.0 * al * np.eye(3)[None, None]) * phi[..., None, None]
    e = np.zeros((basis.nbf, 3))
    e[np.arange(basis.nbf)[is_p], basis.comp[is_p]] = 1.0
    ed = e[None, :, :, None] * d[..., None, :]                   # e_c d^T
    H -= 2.0 * al * g[..., None, None] * (ed + ed.transpose(0, 1, 3, 2))
    return np.ascontiguousarray(H)


def ao_density(phi: np.ndarray, dphi: np.ndarray, P: np.ndarray):
    """rho = sum_{mu nu} P_mu_nu phi_mu phi_nu and its gradient (P symmetric), as in the
    definition of the trial density rho^t from P^t (Sec. II.B)."""
    Pphi = phi @ P                                              # (n, nbf)
    rho = np.einsum("nm,nm->n", Pphi, phi)
    grad = 2.0 * np.einsum("nm,nmk->nk", Pphi, dphi)
    return rho, grad


def ao_nuclear_derivatives(basis: AOBasis, P: np.ndarray, phi: np.ndarray, dphi: np.ndarray,
                           d2phi: np.ndarray, atom_of_point: np.ndarray, n_atom: int):
    """d rho_i / d R_{A,c} and d grad rho_i / d R_{A,c} of rho = sum P_mu_nu phi_mu phi_nu at grid
    points that move with their atom, the density matrix held fixed: phi_mu(r_i - R_C(mu)) moves
    by (delta(A, owner of i) - delta(A, C(mu))) d phi_mu / d x_c, so
      rho^a = 2 sum_mu phi^a_mu (P phi)_mu,
      grad rho^a = 2 sum_mu [grad phi^a_mu (P phi)_mu + phi^a_mu (P grad phi)_mu].
    (3 n_atom, n) and (3 n_atom, n, 3), a = 3 A + c."""
    n = phi.shape[0]
    Pphi = phi @ P                                    # (n, nbf)
    Pdphi = np.einsum("mk,nkd->nmd", P, dphi)         # (n, nbf, 3)
    rt = np.zeros((3 * n_atom, n))
    gt = np.zeros((3 * n_atom, n, 3))
    for A in range(n_atom):
        sig = (atom_of_point == A).astype(float)[:, None] - (basis.atom == A).astype(float)[None, :]
        for c in range(3):
            pa = sig * dphi[:, :, c]                  # phi^a (n, nbf)
            ga = sig[..., None] * d2phi[:, :, c, :]   # grad phi^a (n, nbf, 3)
            rt[3 * A + c] = 2.0 * np.einsum("nm,nm->n", pa, Pphi)
            gt[3 * A + c] = 2.0 * (np.einsum("nmd,nm->nd", ga, Pphi)
                                   + np.einsum("nm,nmd->nd", pa, Pdphi))
    return rt, gt


def density_matrix(basis: AOBasis, n_occ: int, rng: np.random.Generator) -> np.ndarray:
    """A random symmetric positive semi-definite P = 2 C C^T with n_occ orbitals."""
    C = rng.normal(size=(basis.nbf, n_occ)) * 0.4
    return 2.0 * C @ C.T


def ao_system(mol: Molecule, n_rad: int, n_ang: int, seed: int, n_trials: int = 0):
    """The molecular grid of mol with an AO-built density: (GridDensity, phi, grad phi, P,
    P^t (n_trials x nbf x nbf, symmetric), rho^t (n_trials x N), grad rho^t)."""
    rng = np.random.default_rng(seed)
    pts, w, own = molecular_grid(mol, n_rad, n_ang)
    basis = ao_basis(mol)
    phi, dphi = ao_values(basis, pts)
    P = density_matrix(basis, max(1, int(mol.charges.sum()) // 2), rng)
    rho, grad = ao_density(phi, dphi, P)
    Pt = rng.normal(size=(n_trials, basis.nbf, basis.nbf)) * 0.1
    Pt = Pt + Pt.transpose(0, 2, 1)
    rt = np.zeros((n_trials, pts.shape[0]))
    gt = np.zeros((n_trials, pts.shape[0], 3))
    for t in range(n_trials):
        rt[t], gt[t] = ao_density(phi, dphi, Pt[t])
    g = GridDensity(pts, w, rho, grad, own, mol)
    return g, phi, dphi, P, Pt, rt, gt


def ao_moving_system(mol: Molecule, n_rad: int, n_ang: int, P: np.ndarray = None, seed: int = 0,
                     rho_min: float = 1e-6, sel: np.ndarray = None):
    """The molecular grid of mol with the AO-built density of the density matrix P (random from
    seed when None) on a fixed subset of the grid points (sel, else those with rho > rho_min), the
    inputs of the nuclear derivatives of the Fock matrix: (GridDensity, phi, grad phi, hess phi,
    basis, P, sel, rho^a, grad rho^a, w^a), the derivatives along a = 3 A + c with the points,
    the weights and the basis moving with the atoms.  Rebuilt at a displaced geometry with the
    same P and sel, the subset holds the same points."""
    pts, w, own = molecular_grid(mol, n_rad, n_ang)
    basis = ao_basis(mol)
    if P is None:
        P = density_matrix(basis, max(1, int(mol.charges.sum()) // 2), np.random.default_rng(seed))
    phi, dphi = ao_values(basis, pts)
    rho, grad = ao_density(phi, dphi, P)
    if sel is None:
        sel = rho > rho_min
    pts, w, own, phi, dphi = pts[sel], w[sel], own[sel], phi[sel], dphi[sel]
    d2phi = ao_second_derivatives(basis, pts)
    g = GridDensity(np.ascontiguousarray(pts), np.ascontiguousarray(w),
                    np.ascontiguousarray(rho[sel]), np.ascontiguousarray(grad[sel]),
                    np.ascontiguousarray(own), mol)
    rt, gt = ao_nuclear_derivatives(basis, P, phi, dphi, d2phi, own, mol.n_atom)
    W = np.ascontiguousarray(weight_directions(mol, n_rad, n_ang)[:, sel])
    return g, np.ascontiguousarray(phi), np.ascontiguousarray(dphi), d2phi, basis, P, sel, rt, gt, W


def config_water(n_rad: int = 30, n_ang: int = 110) -> GridDensity:
    """Water, 30 x 110 points per atom = 9,900 points."""
    return make_system(water(), n_rad, n_ang)


def config_water_hexamer(n_rad: int = 50, n_ang: int = 194, seed: int = SEED_BASE + 1) -> GridDensity:
    """Six rigid waters, 50 x 194 points per atom = 174,600 points (P = 54)."""
    return make_system(water_cluster(np.random.default_rng(seed)), n_rad, n_ang)


def config_chon60(n_rad: int = 75, n_ang: int = 302, seed: int = SEED_BASE + 2,
                  n_atom: int = 60) -> GridDensity:
    """60-atom random CHON molecule, 75 x 302 points per atom = 1,359,000 points (P = 180)."""
    return make_system(random_chon(np.random.default_rng(seed), n_atom), n_rad, n_ang)


def config_batch(n_mol: int = 64, n_rad: int = 50, n_ang: int = 194, seed: int = SEED_BASE + 3,
                 atom_range=(3, 30), workers: int = 1) -> List[GridDensity]:
    """Batch of random CHON molecules with U{3..30} atoms, 50 x 194 points per atom.

    workers > 1 builds the molecules' grids in that many spawned processes (same result)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(atom_range[0], atom_range[1] + 1, size=n_mol)
    mols = [random_chon(rng, int(s)) for s in sizes]
    if workers <= 1:
        return [make_system(m, n_rad, n_ang) for m in mols]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(workers, n_mol)) as pool:
        return pool.starmap(make_system, [(m, n_rad, n_ang) for m in mols], chunksize=1)


def config_cluster24(n_rad: int = 30, n_ang: int = 139, seed: int = SEED_BASE + 4) -> GridDensity:
    """Four 6-atom CHON fragments 3-4 A apart, 30 x 139 points per atom = 100,080 points."""
    return make_system(fragment_cluster(np.random.default_rng(seed)), n_rad, n_ang)


def random_points(n: int, seed: int, spread: float = 2.0, n_atom: int = 2) -> GridDensity:
    """Tiny random system for brute-force tests: a few atoms, n scattered points.

    Points are drawn around the atoms with positive random weights, so every pair
    quantity is generic (no symmetry, no coincident points).
    """
    rng = np.random.default_rng(seed)
    atoms = rng.normal(scale=1.5, size=(n_atom, 3))
    syms = [["O", "C", "N", "H"][k % 4] for k in range(n_atom)]
    mol = Molecule(syms, atoms)
    own = np.sort(rng.integers(0, n_atom, size=n)).astype(np.int32)
    coords = atoms[own] + rng.normal(scale=spread, size=(n, 3)) * 0.5
    weights = rng.uniform(0.05, 0.5, size=n)
    rho, grad = density(mol, coords)
    return GridDensity(coords, weights, rho, grad, own, mol)
