"""Seeded synthetic inputs for the TDDFT-ris path.

This module only produces arrays: geometries, basis/auxiliary shell lists,
Haar-random orthogonal matrices, orbital energies and the MO coefficients
C = S^-1/2 Q built from them.  It contains none of the ris method's
arithmetic (no two-electron integrals, no response kernel, no derivatives);
the overlap matrix S that the MO recipe needs is evaluated here by plain
Gauss-Hermite quadrature of the one-dimensional Gaussian products.

Both the CUDA path and the CPU oracle receive their inputs from here.

Conventions
-----------
* Lengths in bohr (1 Angstrom = 1/0.529177210903 bohr), energies in Hartree.
* A shell is (atom, l, exponent); every shell is one uncontracted cartesian
  primitive.  Cartesian components are ordered lexicographically
  (p: x,y,z; d: xx,xy,xz,yy,yz,zz) and each component is normalised to
  <chi|chi> = 1.
* The auxiliary basis is the minimal ris set: one s Gaussian per atom with
  exponent 0.2/R_A^2 (R_C = 1.32, R_H = 0.59 bohr), optionally one p shell
  of the same exponent on every carbon (the ris auxiliary basis of the
  paper's Sec. 2.2 holds one Gaussian per angular-momentum component per
  atom).  The Coulomb-fitting (J) set carries s (+p on C); the
  exchange-fitting (K) set carries s only (the paper's Sec. 4 uses s and p
  for Coulomb and s only for exchange).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

ANGSTROM = 1.0 / 0.529177210903  # bohr per Angstrom

Z_OF = {"H": 1, "C": 6}

# Even-tempered uncontracted basis of the synthetic workloads.
BASIS = {
    "C": [(0, 0.1 * 4.0 ** k) for k in range(4)]
    + [(1, 0.15 * 4.0 ** k) for k in range(3)]
    + [(2, 0.8)],
    "H": [(0, 0.12 * 4.0 ** k) for k in range(3)] + [(1, 0.75)],
}
RIS_RADIUS = {"C": 1.32, "H": 0.59}  # bohr


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def cart_components(l: int) -> List[Tuple[int, int, int]]:
    """Lexicographic cartesian exponents (x first)."""
    out = []
    for lx in range(l, -1, -1):
        for ly in range(l - lx, -1, -1):
            out.append((lx, ly, l - lx - ly))
    return out


SHELL_DTYPE = np.dtype([("atom", np.int32), ("l", np.int32), ("exp", np.float64)])


@dataclasses.dataclass
class Molecule:
    """A synthetic workload: geometry, basis, aux sets, MOs, orbital energies."""

    name: str
    elements: List[str]
    coords: np.ndarray  # [natm,3] bohr
    shells: np.ndarray  # SHELL_DTYPE
    aux_j: np.ndarray  # SHELL_DTYPE
    aux_k: np.ndarray  # SHELL_DTYPE
    nocc: int
    C: Optional[np.ndarray] = None  # [nao, nmo] row-major
    mo_energy: Optional[np.ndarray] = None  # [nmo]

    @property
    def natm(self) -> int:
        return len(self.elements)

    @property
    def nao(self) -> int:
        return int(sum(ncart(int(l)) for l in self.shells["l"]))

    @property
    def nmo(self) -> int:
        return self.nao if self.C is None else int(self.C.shape[1])

    @property
    def nvir(self) -> int:
        return self.nmo - self.nocc

    def naux(self, which: str = "J") -> int:
        s = self.aux_j if which == "J" else self.aux_k
        return int(sum(ncart(int(l)) for l in s["l"]))


# ----------------------------------------------------------------- geometry

def chain_geometry(n: int) -> Tuple[List[str], np.ndarray]:
    """All-trans zigzag C_nH_{n+2} in the xy plane (Angstrom in, bohr out).

    C0 at the origin; bond vectors alternate 1.40*(cos30, +-sin30) A; each
    inner C has one H on the outward bisector; each terminal C has two H at
    +-120 degrees from its C-C bond; C-H 1.09 A.
    """
    assert n >= 2
    cc, ch = 1.40, 1.09
    c30, s30 = math.cos(math.radians(30)), math.sin(math.radians(30))
    cpos = [np.zeros(3)]
    for k in range(n - 1):
        sgn = 1.0 if k % 2 == 0 else -1.0
        cpos.append(cpos[-1] + cc * np.array([c30, sgn * s30, 0.0]))
    hpos = []
    for k in range(n):
        if 0 < k < n - 1:
            u1 = cpos[k - 1] - cpos[k]
            u2 = cpos[k + 1] - cpos[k]
            b = -(u1 / np.linalg.norm(u1) + u2 / np.linalg.norm(u2))
            hpos.append(cpos[k] + ch * b / np.linalg.norm(b))
        else:
            nb = cpos[1] if k == 0 else cpos[n - 2]
            d = (nb - cpos[k]) / np.linalg.norm(nb - cpos[k])
            for ang in (120.0, -120.0):
                a = math.radians(ang)
                r = np.array([d[0] * math.cos(a) - d[1] * math.sin(a),
                              d[0] * math.sin(a) + d[1] * math.cos(a), 0.0])
                hpos.append(cpos[k] + ch * r)
    elements = ["C"] * n + ["H"] * len(hpos)
    xyz = np.array(cpos + hpos) * ANGSTROM
    return elements, xyz


def flake_geometry(radius_ang: float) -> Tuple[List[str], np.ndarray]:
    """Honeycomb C sites (C-C 1.42 A) within radius of a hexagon centre at the
    origin, H at 1.09 A on the outward bisector of every 2-coordinated C."""
    a = 1.42
    ch = 1.09
    t1 = math.sqrt(3) * a * np.array([math.cos(math.radians(30)), math.sin(math.radians(30)), 0.0])
    t2 = math.sqrt(3) * a * np.array([0.0, 1.0, 0.0])
    verts = [a * np.array([math.cos(math.radians(60 * k)), math.sin(math.radians(60 * k)), 0.0])
             for k in range(6)]
    nmax = int(radius_ang / (math.sqrt(3) * a)) + 3
    sites = {}
    for i in range(-nmax, nmax + 1):
        for j in range(-nmax, nmax + 1):
            c = i * t1 + j * t2
            for v in verts:
                p = c + v
                if np.linalg.norm(p) <= radius_ang + 1e-6:
                    key = (round(p[0], 4), round(p[1], 4))
                    sites[key] = p
    keys = sorted(sites.keys(), key=lambda k: (round(math.hypot(*k), 4), math.atan2(k[1], k[0])))
    cpos = np.array([sites[k] for k in keys])
    d = np.linalg.norm(cpos[:, None, :] - cpos[None, :, :], axis=-1)
    nbr = (d < a + 0.1) & (d > 1e-6)
    deg = nbr.sum(1)
    if np.any(deg < 2):
        raise ValueError("flake has a dangling carbon")
    hpos = []
    for k in range(len(cpos)):
        if deg[k] == 2:
            nb = np.where(nbr[k])[0]
            u = sum((cpos[j] - cpos[k]) / np.linalg.norm(cpos[j] - cpos[k]) for j in nb)
            hpos.append(cpos[k] - ch * u / np.linalg.norm(u))
    elements = ["C"] * len(cpos) + ["H"] * len(hpos)
    xyz = np.vstack([cpos, np.array(hpos).reshape(-1, 3)]) * ANGSTROM
    return elements, xyz


def haar_rotation(rng: np.random.Generator) -> np.ndarray:
    q = haar_orthogonal(3, rng)
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def packed_chains(ncopy: int, n: int, box_ang: float, min_dist_ang: float,
                  rng: np.random.Generator) -> Tuple[List[str], np.ndarray]:
    """ncopy chains C_nH_{n+2}, each Haar-rotated about its centroid and
    centred uniformly in [0, box]^3 A, redrawn while any atom is closer than
    min_dist to an atom already placed."""
    el0, xyz0 = chain_geometry(n)
    xyz0 = xyz0 / ANGSTROM
    xyz0 = xyz0 - xyz0.mean(0)
    elements: List[str] = []
    placed = np.zeros((0, 3))
    for _ in range(ncopy):
        for _attempt in range(100000):
            r = haar_rotation(rng)
            t = rng.uniform(0.0, box_ang, size=3)
            x = xyz0 @ r.T + t
            if placed.shape[0] == 0:
                break
            dmin = np.min(np.linalg.norm(x[:, None, :] - placed[None, :, :], axis=-1))
            if dmin >= min_dist_ang:
                break
        else:
            raise RuntimeError("could not place chain")
        placed = np.vstack([placed, x])
        elements += el0
    return elements, placed * ANGSTROM


# ----------------------------------------------------------------- basis

def build_shells(elements: Sequence[str]) -> np.ndarray:
    rows = []
    for ia, el in enumerate(elements):
        for l, e in BASIS[el]:
            rows.append((ia, l, e))
    return np.array(rows, dtype=SHELL_DTYPE)


def build_aux(elements: Sequence[str], p_on_heavy: bool) -> np.ndarray:
    rows = []
    for ia, el in enumerate(elements):
        e = 0.2 / RIS_RADIUS[el] ** 2
        rows.append((ia, 0, e))
        if p_on_heavy and el != "H":
            rows.append((ia, 1, e))
    return np.array(rows, dtype=SHELL_DTYPE)


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a standard normal matrix with
    the columns of Q multiplied by sign(diag R)."""
    a = rng.standard_normal((n, n))
    q, r = np.linalg.qr(a)
    return q * np.sign(np.diag(r))[None, :]


def orbital_energies(nocc: int, nvir: int, rng: np.random.Generator) -> np.ndarray:
    eo = np.sort(rng.uniform(-1.0, -0.3, size=nocc))
    ev = np.sort(rng.uniform(0.0, 2.0, size=nvir))
    return np.concatenate([eo, ev])


# ----------------------------------------------------------------- overlap (input recipe only)

_GH_X, _GH_W = np.polynomial.hermite.hermgauss(12)


def _norm(l: Tuple[int, int, int], a: float) -> float:
    def df(n):  # (2n-1)!!
        r = 1.0
        for k in range(1, 2 * n, 2):
            r *= k
        return r
    L = sum(l)
    return math.sqrt((2 * a / math.pi) ** 1.5 * (4 * a) ** L / (df(l[0]) * df(l[1]) * df(l[2])))


def _ov1d(i: int, j: int, a: float, b: float, A: float, B: float) -> float:
    p = a + b
    P = (a * A + b * B) / p
    pref = math.exp(-a * b / p * (A - B) ** 2) / math.sqrt(p)
    x = _GH_X / math.sqrt(p) + P
    return pref * float(np.sum(_GH_W * (x - A) ** i * (x - B) ** j))


def overlap_matrix(coords: np.ndarray, shells: np.ndarray) -> np.ndarray:
    """AO overlap S by Gauss-Hermite quadrature (exact for these polynomials)."""
    atom, cart, expo, norm = [], [], [], []
    for s in shells:
        for c in cart_components(int(s["l"])):
            atom.append(int(s["atom"]))
            cart.append(c)
            expo.append(float(s["exp"]))
            norm.append(_norm(c, float(s["exp"])))
    cart = np.array(cart, dtype=np.float64)
    a = np.array(expo)
    pos = coords[np.array(atom)]
    p = a[:, None] + a[None, :]
    S = np.outer(norm, norm)
    for d in range(3):
        A = pos[:, d]
        P = (a[:, None] * A[:, None] + a[None, :] * A[None, :]) / p
        pref = np.exp(-a[:, None] * a[None, :] / p * (A[:, None] - A[None, :]) ** 2) / np.sqrt(p)
        x = _GH_X[None, None, :] / np.sqrt(p)[:, :, None] + P[:, :, None]
        fa = (x - A[:, None, None]) ** cart[:, d][:, None, None]
        fb = (x - A[None, :, None]) ** cart[:, d][None, :, None]
        S *= pref * np.einsum("k,ijk->ij", _GH_W, fa * fb)
    return 0.5 * (S + S.T)


def lowdin_mo(S: np.ndarray, Q: np.ndarray, min_eig: float = 1e-10) -> np.ndarray:
    w, U = np.linalg.eigh(S)
    if w[0] < min_eig:
        raise ValueError(f"overlap nearly singular: lambda_min={w[0]:.3e}")
    return (U * (w ** -0.5)[None, :]) @ U.T @ Q


# ----------------------------------------------------------------- workloads

def n_electrons(elements: Sequence[str]) -> int:
    return sum(Z_OF[e] for e in elements)


def canonical_mo(S: np.ndarray, rng: np.random.Generator, cutoff: float) -> np.ndarray:
    """C = U_k diag(lambda_k^-1/2) Q over the overlap eigenpairs with
    lambda_k > cutoff (canonical orthogonalisation), Q Haar-orthogonal of the
    kept dimension: orthonormal MOs, nmo <= nao, with |C| <= cutoff^-1/2."""
    w, U = np.linalg.eigh(S)
    keep = w > cutoff
    Q = haar_orthogonal(int(keep.sum()), rng)
    return (U[:, keep] * (w[keep] ** -0.5)[None, :]) @ Q


def make_molecule(name: str, elements: List[str], coords: np.ndarray, seed: int,
                  p_aux: bool, with_mo: bool = True, lindep: float = 0.0) -> Molecule:
    """lindep = 0: Loewdin MOs S^-1/2 Q over all nao AOs; lindep > 0: canonical
    MOs dropping overlap eigenvalues <= lindep (fewer virtual orbitals)."""
    shells = build_shells(elements)
    aux_j = build_aux(elements, p_aux)
    aux_k = build_aux(elements, False)
    nocc = n_electrons(elements) // 2
    mol = Molecule(name, list(elements), np.asarray(coords, dtype=np.float64), shells,
                   aux_j, aux_k, nocc)
    if with_mo:
        rng = np.random.default_rng(seed)
        nao = mol.nao
        S = overlap_matrix(mol.coords, shells)
        if lindep > 0:
            C = canonical_mo(S, rng, lindep)
        else:
            C = lowdin_mo(S, haar_orthogonal(nao, rng))
        eps = orbital_energies(nocc, C.shape[1] - nocc, rng)
        mol.C = np.ascontiguousarray(C)
        mol.mo_energy = eps
    return mol


def chain_molecule(n: int, seed: int, p_aux: bool, with_mo: bool = True) -> Molecule:
    el, xyz = chain_geometry(n)
    return make_molecule(f"C{n}H{n + 2}", el, xyz, seed, p_aux, with_mo)


def flake_molecule(radius_ang: float, seed: int, with_mo: bool = True) -> Molecule:
    el, xyz = flake_geometry(radius_ang)
    nc = el.count("C")
    return make_molecule(f"C{nc}H{len(el) - nc}", el, xyz, seed, True, with_mo)


def workload(idx: int, with_mo: bool = True) -> Molecule:
    """The five synthetic workloads.

    0: C4H6 chain, s-only aux, nocc 15                (tiny, oracle-complete)
    1: C20H22 chain, s+p(C) J-aux, s K-aux            (throughput workload)
    2: C54H18 flake (7 A), s+p(C) J-aux               (RPA workload)
    3: 12 x C20H22 packed in a 40 A cube               (large streamed workload)
    4: serving molecules are built per request (see serving_molecule)
    """
    seed = 1001 + idx
    if idx == 0:
        return chain_molecule(4, seed, p_aux=False, with_mo=with_mo)
    if idx == 1:
        return chain_molecule(20, seed, p_aux=True, with_mo=with_mo)
    if idx == 2:
        return flake_molecule(7.0, seed, with_mo=with_mo)
    if idx == 3:
        rng = np.random.default_rng(seed + 1_000_000)
        el, xyz = packed_chains(12, 20, 40.0, 3.0, rng)
        return make_molecule("12xC20H22", el, xyz, seed, True, with_mo)
    raise ValueError(idx)


def packed_cutdown(ncopy: int = 2, with_mo: bool = True) -> Molecule:
    """The first ncopy chains of the packed 12 x C20H22 workload (same seeds and
    placement draws, so the chains coincide with the first ncopy there)."""
    seed = 1001 + 3
    rng = np.random.default_rng(seed + 1_000_000)
    el, xyz = packed_chains(ncopy, 20, 40.0, 3.0, rng)
    return make_molecule(f"{ncopy}xC20H22", el, xyz, seed, True, with_mo)


# Overlap-eigenvalue cutoff of the serving molecules' MOs.  Their C stays fixed
# along a trajectory while the geometry moves by 0.05 A per component; with
# Loewdin MOs over the near-dependent combinations of this basis C^T S C then
# ranges over [0.01, 550] for the flakes, and the response matrix acquires
# spurious large negative eigenvalues.  Dropping eigenvalues <= 1e-2 keeps
# C^T S C within about [0.17, 3.3].
SERVING_LINDEP = 1e-2


def serving_molecule(kind: str, size: float, seed: int) -> Molecule:
    if kind == "chain":
        el, xyz = chain_geometry(int(size))
        return make_molecule(f"C{int(size)}H{int(size) + 2}", el, xyz, seed, True,
                             lindep=SERVING_LINDEP)
    el, xyz = flake_geometry(float(size))
    nc = el.count("C")
    return make_molecule(f"C{nc}H{len(el) - nc}", el, xyz, seed, True, lindep=SERVING_LINDEP)


def perturb(coords: np.ndarray, sigma_ang: float, rng: np.random.Generator) -> np.ndarray:
    return coords + rng.normal(0.0, sigma_ang * ANGSTROM, size=coords.shape)


def random_amplitudes(nstate: int, nocc: int, nvir: int, seed: int) -> np.ndarray:
    """Normalised random amplitude vectors [nstate][nocc][nvir] (for operator tests)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nstate, nocc, nvir))
    return x / np.linalg.norm(x.reshape(nstate, -1), axis=1)[:, None, None]
