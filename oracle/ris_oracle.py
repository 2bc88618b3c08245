"""TDDFT-ris oracle: plain, slow, FP64 CPU reference of the ris path.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark import this module.  It shares no code with the
CUDA library (its integrals come from ris_ints.c, an Obara-Saika
implementation; the CUDA path uses McMurchie-Davidson), and it never imports
the product package.  Inputs are plain numpy arrays.

What each part follows
----------------------
* Casida problem, Eq. (casida) with A and B of Eqs. (A_matrix), (B_matrix),
  closed-shell singlet: A_ia,jb = (e_a - e_i) d_ij d_ab + 2 (ia|jb)_J
  - c_x (ij|ab)_K and B_ia,jb = 2 (ia|jb)_J - c_x (ib|ja)_K, the factor 2 on
  the Coulomb term being the singlet spin sum and the pure XC kernel dropped
  as in Eq. (ris).
* RI with the minimal auxiliary basis, Eq. (g_modified):
  (pq|rs)_X = sum_AB (pq|A) (M_X^-1)_AB (B|rs), M_AB = (A|B), taken
  literally (M^-1 by a linear solve).
* Pair energy at fixed MO coefficients, orbital energies and amplitudes,
  E_IJ = 1/2 [R_I (A+B) R_J + L_I (A-B) L_J], R = X+Y, L = X-Y (Appendix A,
  R_I and L_I); TDA is the same with Y = 0 (Sec. 3).
* Gradient g_I = dE_II/dR and derivative coupling
  g_IJ = (dE_IJ/dR)/(E_J - E_I): the <g^{ris,(xi)}; Gamma> terms of
  Eqs. (gI_xi_ris) and (gIJ_xi_ris), with the derivative of the RI integral
  taken term by term as in the RI derivative formula closing Sec. 2.2:
  (pq|A)^xi M^-1 (B|rs) + (pq|A) M^-1 (B|rs)^xi - (pq|A) M^-1 M^xi M^-1 (B|rs).
  Computed one nuclear coordinate at a time from AO derivative integrals
  transformed to the MO blocks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libris_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ris_ints.c (plain gcc, OpenMP)."""
    src = os.path.join(_HERE, "ris_ints.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_boys.restype = ctypes.c_double
        L.oracle_boys.argtypes = [ctypes.c_int, ctypes.c_double]
        L.oracle_int3c.argtypes = [dp, ctypes.c_int, ip, ip, dp, ctypes.c_int, ip, ip, dp, dp]
        L.oracle_int2c.argtypes = [dp, ctypes.c_int, ip, ip, dp, dp]
        L.oracle_int3c_deriv_atom.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip, ip, dp,
                                              ctypes.c_int, ip, ip, dp, dp]
        L.oracle_int2c_deriv_atom.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip, ip, dp, dp]
        L.oracle_overlap.argtypes = [dp, ctypes.c_int, ip, ip, dp, dp]
        L.oracle_int3c_triple.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_int,
                                          ctypes.c_double, dp, ctypes.c_int, ctypes.c_double,
                                          dp, dp]
        L.oracle_int3c_triple_deriv.argtypes = L.oracle_int3c_triple.argtypes
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _ncart(l):
    return (l + 1) * (l + 2) // 2


class _Shells:
    def __init__(self, shells):
        self.atom = np.ascontiguousarray(shells["atom"], dtype=np.int32)
        self.l = np.ascontiguousarray(shells["l"], dtype=np.int32)
        self.ex = np.ascontiguousarray(shells["exp"], dtype=np.float64)
        self.n = len(self.atom)
        self.nfun = int(sum(_ncart(int(l)) for l in self.l))
        self.fun_atom = np.concatenate([[a] * _ncart(int(l)) for a, l in zip(self.atom, self.l)]
                                       ).astype(np.int64) if self.n else np.zeros(0, np.int64)


# --------------------------------------------------------------------- integrals

def boys(m: int, T: float) -> float:
    return lib().oracle_boys(int(m), float(T))


def overlap(coords, shells) -> np.ndarray:
    c = np.ascontiguousarray(coords, dtype=np.float64)
    s = _Shells(shells)
    out = np.zeros((s.nfun, s.nfun))
    lib().oracle_overlap(_dp(c), s.n, _ip(s.atom), _ip(s.l), _dp(s.ex), _dp(out))
    return out


def int3c(coords, shells, aux) -> np.ndarray:
    """(mu nu|P) as [nao][nao][naux]."""
    c = np.ascontiguousarray(coords, dtype=np.float64)
    s, a = _Shells(shells), _Shells(aux)
    out = np.zeros((s.nfun, s.nfun, a.nfun))
    lib().oracle_int3c(_dp(c), s.n, _ip(s.atom), _ip(s.l), _dp(s.ex), a.n, _ip(a.atom),
                       _ip(a.l), _dp(a.ex), _dp(out))
    return out


def int2c(coords, aux) -> np.ndarray:
    c = np.ascontiguousarray(coords, dtype=np.float64)
    a = _Shells(aux)
    out = np.zeros((a.nfun, a.nfun))
    lib().oracle_int2c(_dp(c), a.n, _ip(a.atom), _ip(a.l), _dp(a.ex), _dp(out))
    return out


def int3c_deriv_atom(atom: int, coords, shells, aux) -> np.ndarray:
    """d(mu nu|P)/dR_atom as [3][nao][nao][naux]."""
    c = np.ascontiguousarray(coords, dtype=np.float64)
    s, a = _Shells(shells), _Shells(aux)
    out = np.zeros((3, s.nfun, s.nfun, a.nfun))
    lib().oracle_int3c_deriv_atom(int(atom), _dp(c), s.n, _ip(s.atom), _ip(s.l), _dp(s.ex),
                                  a.n, _ip(a.atom), _ip(a.l), _dp(a.ex), _dp(out))
    return out


def int2c_deriv_atom(atom: int, coords, aux) -> np.ndarray:
    c = np.ascontiguousarray(coords, dtype=np.float64)
    a = _Shells(aux)
    out = np.zeros((3, a.nfun, a.nfun))
    lib().oracle_int2c_deriv_atom(int(atom), _dp(c), a.n, _ip(a.atom), _ip(a.l), _dp(a.ex),
                                  _dp(out))
    return out


def int3c_triple(la, alpha, A, lb, beta, B, lc, gamma, Cc, deriv=False) -> np.ndarray:
    """Normalised integrals of one primitive shell triple: [na][nb][nc], or with
    deriv=True the derivatives w.r.t. each centre: [3 centres][3][na][nb][nc]."""
    A, B, Cc = (np.ascontiguousarray(v, dtype=np.float64) for v in (A, B, Cc))
    n = _ncart(la) * _ncart(lb) * _ncart(lc)
    out = np.zeros(9 * n if deriv else n)
    f = lib().oracle_int3c_triple_deriv if deriv else lib().oracle_int3c_triple
    f(la, alpha, _dp(A), lb, beta, _dp(B), lc, gamma, _dp(Cc), _dp(out))
    shp = (_ncart(la), _ncart(lb), _ncart(lc))
    return out.reshape((3, 3) + shp) if deriv else out.reshape(shp)


# --------------------------------------------------------------------- ris model

def phase_fix(X: np.ndarray) -> np.ndarray:
    """Sign of each state so that its largest-magnitude element is positive
    (ties: smallest flat index)."""
    X = np.array(X, copy=True)
    flat = X.reshape(X.shape[0], -1)
    for k in range(flat.shape[0]):
        j = int(np.argmax(np.abs(flat[k])))
        if flat[k, j] < 0:
            flat[k] *= -1.0
    return flat.reshape(X.shape)


def phase_align(X: np.ndarray, X_prev: np.ndarray, ndet: int = 5):
    """Phase tracking between consecutive geometries of a path (Sec. 2, the
    phase of the excited states along a geometric path): for each state the
    sign of its overlap with the previous step's state, taken over the ndet
    most dominant determinants of the previous state (largest |X_prev|
    elements; equal magnitudes ordered by flat index), decides whether the
    new state is flipped.  Returns the signs (+1 keep, -1 flip; a zero
    overlap keeps) and the aligned X.  Plain loops over states."""
    X = np.asarray(X, dtype=np.float64)
    Xp = np.asarray(X_prev, dtype=np.float64)
    ns = X.shape[0]
    signs = np.ones(ns, dtype=np.int32)
    out = np.array(X, copy=True)
    for k in range(ns):
        xp = Xp[k].ravel()
        x = X[k].ravel()
        mag = np.abs(xp)
        dominant = sorted(range(mag.size), key=lambda i: (-mag[i], i))[:ndet]
        overlap = 0.0
        for i in dominant:
            overlap += x[i] * xp[i]
        if overlap < 0.0:
            signs[k] = -1
            out[k] *= -1.0
    return signs, out


class RisOracle:
    """FP64 TDDFT-ris at fixed MO coefficients, orbital energies and amplitudes."""

    def __init__(self, coords, shells, aux_j, aux_k, C, mo_energy, nocc: int,
                 cx: float = 0.25, metric_inverse: str = "solve"):
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.shells, self.aux_j, self.aux_k = shells, aux_j, aux_k
        self.C = np.ascontiguousarray(C, dtype=np.float64)
        self.eps = np.asarray(mo_energy, dtype=np.float64)
        self.nocc = int(nocc)
        self.nao, self.nmo = self.C.shape
        self.nvir = self.nmo - self.nocc
        self.cx = float(cx)
        self.metric_inverse = metric_inverse
        self.natm = self.coords.shape[0]
        self.Co = self.C[:, :self.nocc]
        self.Cv = self.C[:, self.nocc:]
        self.de = (self.eps[self.nocc:][None, :] - self.eps[:self.nocc][:, None])  # [i][a]
        self._setup()

    def _inverse(self, M):
        """M^-1 of Eq. (g_modified).  The RI integral does not depend on how
        the inverse is formed; the routes differ only in rounding:
        "solve" (LU with partial pivoting, the default), "cholesky"
        (L^-T L^-1 from M = L L^T) or "eigh" (V diag(1/lambda) V^T)."""
        n = M.shape[0]
        if self.metric_inverse == "solve":
            return np.linalg.solve(M, np.eye(n))
        if self.metric_inverse == "cholesky":
            L = np.linalg.cholesky(M)
            Li = np.linalg.solve(L, np.eye(n))
            return Li.T @ Li
        if self.metric_inverse == "eigh":
            w, V = np.linalg.eigh(M)
            return (V / w[None, :]) @ V.T
        raise ValueError(self.metric_inverse)

    # -- integrals in the MO blocks
    def _mo3(self, T, left, right):
        """sum_mu,nu left_mu,p right_nu,q T_mu,nu,P -> [p][q][P]."""
        h = np.tensordot(left, T, axes=([0], [0]))  # [p][nu][P]
        return np.einsum("pnP,nq->pqP", h, right, optimize=True)

    def _setup(self):
        c = self.coords
        self.TJ = int3c(c, self.shells, self.aux_j)
        self.TK = int3c(c, self.shells, self.aux_k)
        self.MJ = int2c(c, self.aux_j)
        self.MK = int2c(c, self.aux_k)
        self.MJinv = self._inverse(self.MJ)
        self.MKinv = self._inverse(self.MK)
        Co, Cv = self.Co, self.Cv
        self.ovJ = self._mo3(self.TJ, Co, Cv)  # (ia|P)_J
        self.ooK = self._mo3(self.TK, Co, Co)  # (ij|P)_K
        self.vvK = self._mo3(self.TK, Cv, Cv)  # (ab|P)_K
        self.ovK = self._mo3(self.TK, Co, Cv)  # (ia|P)_K

    # -- four-index RI blocks as operators
    def _coul(self, U, V, ov1, ov2, Minv):
        """sum U_ia V_jb (ia|A) Minv_AB (B|jb) with separate 3c tensors per side."""
        u = np.tensordot(U, ov1, axes=([0, 1], [0, 1]))
        v = np.tensordot(V, ov2, axes=([0, 1], [0, 1]))
        return u @ Minv @ v

    def apply_A(self, X: np.ndarray) -> np.ndarray:
        """TDA A applied to X [n][nocc][nvir] (Eq. A_matrix with the ris kernel)."""
        out = np.empty_like(X)
        cvv = np.tensordot(self.vvK, self.MKinv, axes=([2], [0]))  # [a][b][P]
        for k in range(X.shape[0]):
            x = X[k]
            w = self.MJinv @ np.tensordot(x, self.ovJ, axes=([0, 1], [0, 1]))
            coul = np.tensordot(self.ovJ, w, axes=([2], [0]))
            t = np.tensordot(x, cvv, axes=([1], [1]))                 # [j][a][P]
            exch = np.tensordot(self.ooK, t, axes=([1, 2], [0, 2]))   # [i][a]
            out[k] = self.de * x + 2.0 * coul - self.cx * exch
        return out

    def apply_ApB_AmB(self, Z: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
        """(A + B) Z and (A - B) Z for Z [n][nocc][nvir] (Eqs. A_matrix,
        B_matrix with the ris kernel): A + B = D + 4 (ia|jb)_J
        - c_x [(ij|ab)_K + (ib|ja)_K], A - B = D - c_x [(ij|ab)_K - (ib|ja)_K].
        Vectors are taken eight at a time (each term one tensor contraction)."""
        if not hasattr(self, "_cvv"):
            self._cvv = np.tensordot(self.vvK, self.MKinv, axes=([2], [0]))   # [a][b][Q]
            self._cov = np.tensordot(self.ovK, self.MKinv, axes=([2], [0]))   # [j][a][Q]
        P = np.empty_like(Z)
        M = np.empty_like(Z)
        for k0 in range(0, Z.shape[0], 8):
            z = Z[k0:k0 + 8]
            w = np.tensordot(z, self.ovJ, axes=([1, 2], [0, 1])) @ self.MJinv       # [k][P]
            coul = np.tensordot(w, self.ovJ, axes=([1], [2]))                        # [k][i][a]
            t = np.tensordot(z, self._cvv, axes=([2], [1]))                          # [k][j][a][Q]
            kx = np.tensordot(t, self.ooK, axes=([1, 3], [1, 2])).transpose(0, 2, 1)  # (ij|ab) z_jb
            u = np.tensordot(z, self.ovK, axes=([2], [1]))                           # [k][j][i][Q]
            kb = np.tensordot(u, self._cov, axes=([1, 3], [0, 2]))                   # (ib|ja) z_jb
            P[k0:k0 + 8] = self.de * z + 4.0 * coul - self.cx * (kx + kb)
            M[k0:k0 + 8] = self.de * z - self.cx * (kx - kb)
        return P, M

    def rpa_davidson(self, nstates: int, tol: float = 1e-10, max_iter: int = 200,
                     max_space: Optional[int] = None):
        """Lowest RPA excitations by a plain Davidson on the Casida problem
        (Eq. casida) in its symmetric form: omega^2 are the eigenvalues of
        (A-B)^1/2 (A+B) (A-B)^1/2, since (A+B) R = omega L and
        (A-B) L = omega R with R = X+Y, L = X-Y.  One orthonormal basis V
        spans both R and L; the projected problem is the symmetric
        eigenproblem of Mm^1/2 P Mm^1/2 with P = V^T (A+B) V and
        Mm = V^T (A-B) V (the dense form of rpa_dense, in the subspace).
        New directions: both residuals divided by (D - omega), D the
        orbital-energy differences.  Converged when both residuals
        (A+B) R - omega L and (A-B) L - omega R have 2-norm <= tol per state,
        R = X+Y and L = X-Y normalised so that R . L = 1 (sum X^2 - Y^2 = 1).
        Returns omega [nstates], X, Y [nstates][nocc][nvir] (largest |X|
        element positive) and the iteration count."""
        o, v = self.nocc, self.nvir
        n = o * v
        de = self.de.reshape(-1)
        nb = nstates + min(nstates, 8)
        max_space = max_space or max(20 * nstates, 4 * nb)
        order = np.lexsort((np.arange(n), de))
        V = np.zeros((nb, n))
        for k in range(nb):
            V[k, order[k]] = 1.0
        P_, M_ = self.apply_ApB_AmB(V.reshape(nb, o, v))
        PV, MV = P_.reshape(nb, n), M_.reshape(nb, n)
        for it in range(max_iter):
            Ps = V @ PV.T
            Ms = V @ MV.T
            Ps, Ms = 0.5 * (Ps + Ps.T), 0.5 * (Ms + Ms.T)
            wm, Um = np.linalg.eigh(Ms)
            if wm[0] <= 0:
                raise RuntimeError("projected A-B not positive definite")
            Sh = (Um * np.sqrt(wm)[None, :]) @ Um.T                # Mm^1/2
            w2, T = np.linalg.eigh(Sh @ Ps @ Sh)
            om = np.sqrt(w2[:nstates])
            # subspace R (= X+Y) and L (= X-Y) with R . L = 1
            r = (Sh @ T[:, :nstates]) / np.sqrt(om)[None, :]
            l = (Ps @ r) / om[None, :]
            R, L = r.T @ V, l.T @ V
            res1 = r.T @ PV - om[:, None] * L        # (A+B) R - omega L
            res2 = l.T @ MV - om[:, None] * R        # (A-B) L - omega R
            rn = np.maximum(np.linalg.norm(res1, axis=1), np.linalg.norm(res2, axis=1))
            if np.all(rn <= tol):
                X = (0.5 * (R + L)).reshape(nstates, o, v)
                Y = (0.5 * (R - L)).reshape(nstates, o, v)
                for k in range(nstates):
                    j = int(np.argmax(np.abs(X[k].ravel())))
                    if X[k].ravel()[j] < 0:
                        X[k] *= -1.0
                        Y[k] *= -1.0
                return om, X, Y, it
            new = []
            for k in range(nstates):
                if rn[k] <= tol:
                    continue
                den = de - om[k]
                den = np.where(np.abs(den) < 1e-8, np.copysign(1e-8, den), den)
                new.append(res1[k] / den)
                new.append(res2[k] / den)
            new = np.array(new)
            if V.shape[0] + new.shape[0] > max_space:
                # restart on span{R, L}; the products follow linearly
                q, _ = np.linalg.qr(np.vstack([R, L]).T)
                Cm = q.T @ V.T
                V, PV, MV = Cm @ V, Cm @ PV, Cm @ MV
            for _ in range(2):
                new = new - (new @ V.T) @ V
            q, rr = np.linalg.qr(new.T)
            q = q.T[np.abs(np.diag(rr)) > 1e-8 * np.max(np.abs(np.diag(rr)))]
            for _ in range(2):
                q = q - (q @ V.T) @ V
                q = q / np.linalg.norm(q, axis=1)[:, None]
            P_, M_ = self.apply_ApB_AmB(q.reshape(-1, o, v))
            V = np.vstack([V, q])
            PV = np.vstack([PV, P_.reshape(-1, n)])
            MV = np.vstack([MV, M_.reshape(-1, n)])
        raise RuntimeError("oracle RPA Davidson did not converge")

    def dense_AB(self) -> Tuple[np.ndarray, np.ndarray]:
        """Dense A and B over the ia pair index (small systems only)."""
        o, v = self.nocc, self.nvir
        J = np.einsum("iaP,PQ,jbQ->iajb", self.ovJ, self.MJinv, self.ovJ, optimize=True)
        Kx = np.einsum("ijP,PQ,abQ->iajb", self.ooK, self.MKinv, self.vvK, optimize=True)
        Kb = np.einsum("ibP,PQ,jaQ->iajb", self.ovK, self.MKinv, self.ovK, optimize=True)
        n = o * v
        A = (2.0 * J - self.cx * Kx).reshape(n, n) + np.diag(self.de.reshape(-1))
        B = (2.0 * J - self.cx * Kb).reshape(n, n)
        return A, B

    # -- Z-vector equation with the ris kernel
    def zvector(self, rhs: np.ndarray) -> np.ndarray:
        """Solve (A + B) Z = rhs (Eq. Z_vector with the ris kernel of Eq. ris in
        A + B) by a dense solve; rhs [n][nocc][nvir] (small systems only)."""
        A, B = self.dense_AB()
        n = self.nocc * self.nvir
        R = np.asarray(rhs).reshape(-1, n)
        Z = np.linalg.solve(A + B, R.T).T
        return Z.reshape(np.asarray(rhs).shape)

    def apb_form(self, U, V) -> float:
        """U . (A + B) . V through the integral-level kernels (no dense matrix)."""
        return float(np.sum(self.de * U * V)) + self._kernel_ApB(U, V)

    # -- excitation energies
    def tda_dense(self, nstates: int):
        A, _ = self.dense_AB()
        w, V = np.linalg.eigh(A)
        X = V[:, :nstates].T.reshape(nstates, self.nocc, self.nvir)
        return w[:nstates], phase_fix(X)

    def rpa_dense(self, nstates: int):
        A, B = self.dense_AB()
        ApB, AmB = A + B, A - B
        wm, Um = np.linalg.eigh(AmB)
        if wm[0] <= 0:
            raise ValueError("A-B not positive definite")
        S = (Um * np.sqrt(wm)[None, :]) @ Um.T
        H = S @ ApB @ S
        w2, T = np.linalg.eigh(0.5 * (H + H.T))
        om = np.sqrt(w2[:nstates])
        R = (S @ T[:, :nstates]) / np.sqrt(om)[None, :]
        L = (ApB @ R) / om[None, :]
        X = 0.5 * (R + L)
        Y = 0.5 * (R - L)
        shp = (nstates, self.nocc, self.nvir)
        X, Y = X.T.reshape(shp), Y.T.reshape(shp)
        for k in range(nstates):  # phase by the largest element of X
            j = np.argmax(np.abs(X[k].ravel()))
            if X[k].ravel()[j] < 0:
                X[k] *= -1
                Y[k] *= -1
        return om, X, Y

    def tda_davidson(self, nstates: int, tol: float = 1e-11, max_iter: int = 200,
                     max_space: Optional[int] = None):
        """Plain block Davidson on A (symmetric), FP64; ascending eigenpairs."""
        o, v = self.nocc, self.nvir
        n = o * v
        de = self.de.reshape(-1)
        nb = nstates + min(nstates, 8)
        max_space = max_space or max(20 * nstates, 4 * nb)
        order = np.lexsort((np.arange(n), de))
        V = np.zeros((nb, n))
        for k in range(nb):
            V[k, order[k]] = 1.0
        AV = self.apply_A(V.reshape(nb, o, v)).reshape(nb, n)
        for it in range(max_iter):
            H = V @ AV.T
            w, s = np.linalg.eigh(0.5 * (H + H.T))
            w, s = w[:nstates], s[:, :nstates]
            Xr = s.T @ V
            R = s.T @ AV - w[:, None] * Xr
            rn = np.linalg.norm(R, axis=1)
            if np.all(rn <= tol):
                X = Xr.reshape(nstates, o, v)
                return w, phase_fix(X), it
            new = []
            for k in range(nstates):
                if rn[k] <= tol:
                    continue
                den = de - w[k]
                den = np.where(np.abs(den) < 1e-8, np.copysign(1e-8, den), den)
                new.append(R[k] / den)
            new = np.array(new)
            if V.shape[0] + new.shape[0] > max_space:
                keep = min(2 * nstates + 0, V.shape[0])
                wf, sf = np.linalg.eigh(0.5 * (H + H.T))
                V = sf[:, :keep].T @ V
                AV = sf[:, :keep].T @ AV
            for _ in range(2):
                new = new - (new @ V.T) @ V
            q, _r = np.linalg.qr(new.T)
            q = q.T
            nrm_ok = np.abs(np.diag(_r)) > 1e-8 * np.max(np.abs(np.diag(_r)))
            q = q[nrm_ok]
            for _ in range(2):
                q = q - (q @ V.T) @ V
                q = q / np.linalg.norm(q, axis=1)[:, None]
            V = np.vstack([V, q])
            AV = np.vstack([AV, self.apply_A(q.reshape(-1, o, v)).reshape(-1, n)])
        raise RuntimeError("oracle Davidson did not converge")

    # -- pair energies and their nuclear derivatives (fixed C, eps, amplitudes)
    def pair_energy(self, XI, XJ, YI=None, YJ=None) -> float:
        """E_IJ = 1/2 [R_I (A+B) R_J + L_I (A-B) L_J] without the constant
        orbital-energy part is returned with it included (Delta-eps term)."""
        YI = np.zeros_like(XI) if YI is None else YI
        YJ = np.zeros_like(XJ) if YJ is None else YJ
        RI, RJ, LI, LJ = XI + YI, XJ + YJ, XI - YI, XJ - YJ
        return 0.5 * (self._kernel_ApB(RI, RJ) + self._kernel_AmB(LI, LJ)) + \
            0.5 * (np.sum(self.de * RI * RJ) + np.sum(self.de * LI * LJ))

    def _xk(self, U, V, oo, vv, Minv):
        """sum U_ia V_jb (ij|A) Minv_AB (B|ab)."""
        t = np.tensordot(U, vv, axes=([1], [0]))          # [i][b][Q]
        t = np.tensordot(t, V, axes=([1], [1]))           # [i][Q][j]
        u = np.tensordot(oo, Minv, axes=([2], [0]))       # [i][j][Q]
        return float(np.einsum("ijQ,iQj->", u, t))

    def _bk(self, U, V, ov1, ov2, Minv):
        """sum U_ia V_jb (ib|A) Minv_AB (B|ja)."""
        t = np.tensordot(U, ov2, axes=([1], [1]))         # [i][j][Q]  (sum_a U_ia (ja|Q))
        t2 = np.tensordot(V, ov1, axes=([1], [1]))        # [j][i][P]  (sum_b V_jb (ib|P))
        u = np.tensordot(t2, Minv, axes=([2], [0]))       # [j][i][Q]
        return float(np.einsum("jiQ,ijQ->", u, t))

    def _kernel_ApB(self, U, V):
        return (4.0 * self._coul(U, V, self.ovJ, self.ovJ, self.MJinv)
                - self.cx * (self._xk(U, V, self.ooK, self.vvK, self.MKinv)
                             + self._bk(U, V, self.ovK, self.ovK, self.MKinv)))

    def _kernel_AmB(self, U, V):
        return -self.cx * (self._xk(U, V, self.ooK, self.vvK, self.MKinv)
                           - self._bk(U, V, self.ovK, self.ovK, self.MKinv))

    def pair_energy_derivs(self, pairs: Sequence[Tuple[int, int]], X, Y=None,
                           atoms: Optional[Sequence[int]] = None) -> np.ndarray:
        """dE_IJ/dR_(atom,x) for each pair, [npair][natm][3] (rows of atoms not
        requested stay NaN).  One nuclear coordinate at a time: AO derivative
        integrals -> MO blocks -> RI derivative formula term by term."""
        X = np.asarray(X)
        Y = np.zeros_like(X) if Y is None else np.asarray(Y)
        atoms = range(self.natm) if atoms is None else atoms
        out = np.full((len(pairs), self.natm, 3), np.nan)
        Co, Cv = self.Co, self.Cv
        rpa = bool(np.any(Y != 0))
        for A in atoms:
            dTJ = int3c_deriv_atom(A, self.coords, self.shells, self.aux_j)
            dTK = int3c_deriv_atom(A, self.coords, self.shells, self.aux_k)
            dMJ = int2c_deriv_atom(A, self.coords, self.aux_j)
            dMK = int2c_deriv_atom(A, self.coords, self.aux_k)
            for x in range(3):
                d_ovJ = self._mo3(dTJ[x], Co, Cv)
                d_ooK = self._mo3(dTK[x], Co, Co)
                d_vvK = self._mo3(dTK[x], Cv, Cv)
                d_ovK = self._mo3(dTK[x], Co, Cv) if rpa else None
                dMJinv = -self.MJinv @ dMJ[x] @ self.MJinv
                dMKinv = -self.MKinv @ dMK[x] @ self.MKinv
                for p, (I, J) in enumerate(pairs):
                    RI, RJ = X[I] + Y[I], X[J] + Y[J]
                    LI, LJ = X[I] - Y[I], X[J] - Y[J]
                    # d(ia|jb)_J: (ia|A)^x Minv (B|jb) + (ia|A) Minv (B|jb)^x
                    #             - (ia|A) Minv M^x Minv (B|jb)
                    cJ = (self._coul(RI, RJ, d_ovJ, self.ovJ, self.MJinv)
                          + self._coul(RI, RJ, self.ovJ, d_ovJ, self.MJinv)
                          + self._coul(RI, RJ, self.ovJ, self.ovJ, dMJinv))
                    xk = 0.0
                    # TDA (Y = 0): L = R, so the (L, L) term equals the (R, R) one
                    combos = ((RI, RJ), (LI, LJ)) if rpa else ((RI, RJ),)
                    for (U, V) in combos:
                        xk += (self._xk(U, V, d_ooK, self.vvK, self.MKinv)
                               + self._xk(U, V, self.ooK, d_vvK, self.MKinv)
                               + self._xk(U, V, self.ooK, self.vvK, dMKinv))
                    if not rpa:
                        xk = 2.0 * xk
                    bk = 0.0
                    if rpa:
                        for (U, V, s) in ((RI, RJ, 1.0), (LI, LJ, -1.0)):
                            bk += s * (self._bk(U, V, d_ovK, self.ovK, self.MKinv)
                                       + self._bk(U, V, self.ovK, d_ovK, self.MKinv)
                                       + self._bk(U, V, self.ovK, self.ovK, dMKinv))
                    out[p, A, x] = 0.5 * (4.0 * cJ) - 0.5 * self.cx * (xk + bk)
        return out

    def gradients(self, states, X, Y=None, atoms=None) -> np.ndarray:
        """g_I = dE_II/dR, [n][natm][3] in Hartree/bohr."""
        return self.pair_energy_derivs([(s, s) for s in states], X, Y, atoms)

    def nacs(self, pairs, omega, X, Y=None, atoms=None) -> np.ndarray:
        """g_IJ = (dE_IJ/dR)/(omega_J - omega_I), [npair][natm][3] in 1/bohr."""
        num = self.pair_energy_derivs(pairs, X, Y, atoms)
        den = np.array([omega[J] - omega[I] for (I, J) in pairs])
        return num / den[:, None, None]
