"""FP64 CPU oracle for the SPGM near-field MIMO reconstruction.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  It shares no code with the CUDA path;
the only common module is the seeded input generator.

Operator (Sec. II, Eq. 2) in plain C (`nfm_oracle.c`); everything above it is
plain numpy in FP64, written in the paper's order and notation:

  * data fidelity D(s) = ||y - A s||^2 / (2M)                    (Sec. III, Eq. 4)
  * l1 regulariser R(s) = sum_n |s_n| (complex modulus)          (Sec. III); the extensions that
    Sec. III allows: + (w2/2)||s||^2 (elastic net / Tikhonov) and + w3 sum_g ||s_g||_2 over
    2 x 2 x 1 voxel blocks (sparse-group penalty; its prox is the soft threshold followed by the
    group shrink, pinned against the definition of the prox in the tests)
  * PGM step s <- prox_{alpha R}(s - eta grad D(s)), alpha = lambda eta  (Sec. IV, Eq. 5)
  * SPGM: grad D replaced by the gradient of the mean of B component
    functions D_m(s) = |y_m - (A s)_m|^2 / 2 over a minibatch      (Sec. IV-A, Eq. 6)

Readings where the paper is silent (each also listed in the design notes):
  * complex gradient: grad D_m = conj(A_m)^T (A_m s - y_m), i.e. 2 dD/d(conj s);
    the minibatch gradient is (1/B) A_B^H (A_B s - y_B)
  * prox of alpha |.| on complex z: z * max(0, 1 - alpha/|z|), 0 when |z| <= alpha
  * minibatch = B_p whole TX-RX pairs with all K frequencies, B = B_p K rows,
    drawn without replacement from a per-epoch permutation; a short last chunk
    uses its own B
  * step eta = 1/L with L = lambda_max(A^H A)/M from a seeded power iteration
    (or, where that is too slow, from the bound ||A||_F^2/M >= L)
  * lambda = frac * max_n |(A^H y)_n| / M
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


class _Geom(ctypes.Structure):
    _fields_ = [
        ("T", ctypes.c_int), ("R", ctypes.c_int), ("K", ctypes.c_int),
        ("tx", ctypes.c_void_p), ("rx", ctypes.c_void_p),
        ("freq", ctypes.c_void_p), ("pulse", ctypes.c_void_p),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("nx", ctypes.c_long), ("ny", ctypes.c_long), ("nz", ctypes.c_long),
        ("c", ctypes.c_double),
        ("pos", ctypes.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile the C part with gcc (FP64, no fast-math, no FMA contraction)."""
    src = os.path.join(_HERE, "nfm_oracle.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    import subprocess
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", src, "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [src, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.orc_element.argtypes = [ctypes.POINTER(_Geom), ctypes.c_long, ctypes.c_long, P]
        L.orc_dense.argtypes = [ctypes.POINTER(_Geom), P, ctypes.c_long, P, ctypes.c_long, P]
        L.orc_forward.argtypes = [ctypes.POINTER(_Geom), P, ctypes.c_long, P, ctypes.c_long, P, P]
        L.orc_adjoint.argtypes = [ctypes.POINTER(_Geom), P, ctypes.c_long, P, P, ctypes.c_long, P]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_get_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cplx(z):
    z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
    return z


class Oracle:
    """FP64 operator on one geometry (an `inputs.Geometry`)."""

    def __init__(self, geom, w1: float = 1.0, w2: float = 0.0, w3: float = 0.0):
        """w1, w2, w3: regulariser R(s) = w1 ||s||_1 + (w2/2) ||s||_2^2 + w3 sum_g ||s_g||_2 (w2 = w3 = 0:
        the paper's l1; the groups g are the 2 x 2 x 1 voxel blocks of `voxel_groups`)."""
        self.geom = geom
        self.w1, self.w2, self.w3 = float(w1), float(w2), float(w3)
        self.T, self.R, self.K = geom.T, geom.R, geom.K
        self.P, self.M, self.N = geom.P, geom.M, geom.N
        self._tx = np.ascontiguousarray(geom.tx, dtype=np.float64)
        self._rx = np.ascontiguousarray(geom.rx, dtype=np.float64)
        self._f = np.ascontiguousarray(geom.freq, dtype=np.float64)
        if geom.pulse is None:
            self._p = None
        else:
            p = np.asarray(geom.pulse, dtype=np.complex128)
            self._p = np.ascontiguousarray(np.stack([p.real, p.imag], 1))
        g = geom.grid
        pp = None if self._p is None else _ptr(self._p).value
        if hasattr(g, "xyz"):                 # explicit voxel positions (Sec. II: any set of points r_n)
            self._pos = np.ascontiguousarray(g.xyz, dtype=np.float64)
            self._g = _Geom(self.T, self.R, self.K, _ptr(self._tx).value, _ptr(self._rx).value,
                            _ptr(self._f).value, pp, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, g.N, 1, 1, geom.c,
                            _ptr(self._pos).value)
        else:
            self._pos = None
            self._g = _Geom(self.T, self.R, self.K, _ptr(self._tx).value, _ptr(self._rx).value,
                            _ptr(self._f).value, pp, g.x0, g.y0, g.z0, g.dx, g.dy, g.dz, g.nx, g.ny, g.nz,
                            geom.c, None)

    # ---- index helpers --------------------------------------------------
    def rows_of_pairs(self, pairs) -> np.ndarray:
        """Rows m = pair*K + k of the given pairs, pair-major, frequency-minor."""
        pairs = np.asarray(pairs, dtype=np.int64)
        return (pairs[:, None] * self.K + np.arange(self.K)[None, :]).ravel()

    def all_cols(self) -> np.ndarray:
        return np.arange(self.N, dtype=np.int64)

    # ---- Eq. 2 ------------------------------------------------------------
    def element(self, m: int, n: int) -> complex:
        out = np.zeros(2)
        lib().orc_element(ctypes.byref(self._g), int(m), int(n), _ptr(out))
        return complex(out[0], out[1])

    def dense(self, rows, cols) -> np.ndarray:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        out = np.zeros((rows.size, cols.size, 2))
        lib().orc_dense(ctypes.byref(self._g), _ptr(rows), rows.size, _ptr(cols), cols.size, _ptr(out))
        return out[..., 0] + 1j * out[..., 1]

    # ---- matrix-free operator ---------------------------------------------
    def forward(self, s, rows=None, cols=None) -> np.ndarray:
        """(A s) on the given rows; s holds the values of the given columns."""
        rows = np.arange(self.M, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
        cols = self.all_cols() if cols is None else np.ascontiguousarray(cols, dtype=np.int64)
        s = _cplx(s)
        assert s.shape == (cols.size,)
        y = np.zeros(rows.size, dtype=np.complex128)
        lib().orc_forward(ctypes.byref(self._g), _ptr(rows), rows.size, _ptr(cols), cols.size,
                          _ptr(s.view(np.float64)), _ptr(y.view(np.float64)))
        return y

    def forward_sparse(self, s, rows=None) -> np.ndarray:
        """A s using only the nonzero entries of s (exact: zero terms add nothing)."""
        s = np.asarray(s)
        nz = np.flatnonzero(s)
        return self.forward(s[nz], rows=rows, cols=nz)

    def adjoint(self, r, rows=None, cols=None) -> np.ndarray:
        """(A^H r) on the given columns; r holds the values of the given rows."""
        rows = np.arange(self.M, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
        cols = self.all_cols() if cols is None else np.ascontiguousarray(cols, dtype=np.int64)
        r = _cplx(r)
        assert r.shape == (rows.size,)
        g = np.zeros(cols.size, dtype=np.complex128)
        lib().orc_adjoint(ctypes.byref(self._g), _ptr(rows), rows.size, _ptr(r.view(np.float64)),
                          _ptr(cols), cols.size, _ptr(g.view(np.float64)))
        return g

    # ---- Sec. III / IV --------------------------------------------------
    def data_fidelity(self, y, s) -> float:
        """D(s) = ||y - A s||^2 / (2M)   (Eq. 4)."""
        res = np.asarray(y) - self.forward(s)
        return float(np.vdot(res, res).real) / (2.0 * self.M)

    def regulariser(self, s) -> float:
        """R(s) = w1 sum |s_n| + (w2/2) sum |s_n|^2 + w3 sum_g ||s_g||_2   (Sec. III; l1 when w2 = w3 = 0)."""
        s = np.asarray(s)
        r = self.w1 * float(np.sum(np.abs(s))) + 0.5 * self.w2 * float(np.vdot(s, s).real)
        if self.w3 != 0.0:
            r += self.w3 * float(np.sum(group_norms(s, voxel_groups(self.geom.grid))))
        return r

    def prox(self, z, alpha_eta):
        """prox of (eta lambda) R at z, alpha_eta = eta lambda: the soft threshold of the l1 term, then
        the group shrink of the group term (the prox of the sparse-group penalty is that composition),
        then the 1/(1 + eta lambda w2) scaling of the quadratic term."""
        u = prox_l1(z, alpha_eta * self.w1)
        if self.w3 != 0.0:
            u = prox_group(u, voxel_groups(self.geom.grid), alpha_eta * self.w3)
        return u / (1.0 + alpha_eta * self.w2)

    def objective(self, y, s, lam) -> float:
        """D(s) + lambda R(s)   (Eq. 3, Eq. 4)."""
        return self.data_fidelity(y, s) + lam * self.regulariser(s)

    def full_gradient(self, y, s) -> np.ndarray:
        """grad D(s) = A^H (A s - y) / M."""
        return self.adjoint(self.forward(s) - np.asarray(y)) / self.M

    def minibatch_gradient(self, y, s, pairs) -> np.ndarray:
        """grad of (1/B) sum_{m in batch} D_m(s) = A_B^H (A_B s - y_B) / B   (Eq. 6)."""
        rows = self.rows_of_pairs(pairs)
        res = self.forward(s, rows=rows) - np.asarray(y)[rows]
        return self.adjoint(res, rows=rows) / rows.size

    def rows_gradient(self, y, s, rows) -> np.ndarray:
        """grad of (1/B) sum_{m in rows} D_m(s) = A_rows^H (A_rows s - y_rows) / B   (Eq. 6, any row set)."""
        rows = np.asarray(rows, dtype=np.int64)
        res = self.forward(s, rows=rows) - np.asarray(y)[rows]
        return self.adjoint(res, rows=rows) / rows.size

    def spgm_step_rows(self, y, s, rows, eta, lam) -> np.ndarray:
        """SPGM iteration (Eq. 5) with the minibatch gradient over an explicit row set."""
        return self.prox(s - eta * self.rows_gradient(y, s, rows), lam * eta)

    def pgm_step(self, y, s, eta, lam) -> np.ndarray:
        """One PGM fixed-point iteration (Eq. 5), full batch."""
        return self.prox(s - eta * self.full_gradient(y, s), lam * eta)

    def spgm_step(self, y, s, pairs, eta, lam) -> np.ndarray:
        """One SPGM iteration: Eq. 5 with the minibatch gradient of Eq. 6."""
        return self.prox(s - eta * self.minibatch_gradient(y, s, pairs), lam * eta)

    def spgm_epoch(self, y, s, perm, pairs_per_batch, eta, lam) -> np.ndarray:
        """One pass over a permutation of the pairs in chunks of B_p pairs."""
        perm = np.asarray(perm)
        for c0 in range(0, perm.size, pairs_per_batch):
            s = self.spgm_step(y, s, perm[c0:c0 + pairs_per_batch], eta, lam)
        return s

    def power_iteration(self, v0, iters: int, pairs=None) -> float:
        """Largest eigenvalue L of A^H A / M by power iteration from v0; with `pairs`, L_B of the minibatch
        A_B^H A_B / B (B = len(pairs) K rows), the Lipschitz constant of the Eq. 6 minibatch gradient.

        v <- A_B^H A_B v / B, v <- v / ||v|| for `iters` steps, then the Rayleigh
        quotient L = ||A_B v||^2 / (B ||v||^2).
        """
        rows = None if pairs is None else self.rows_of_pairs(pairs)
        B = self.M if rows is None else rows.size
        v = _cplx(v0).copy()
        v /= np.linalg.norm(v)
        for _ in range(iters):
            v = self.adjoint(self.forward(v, rows=rows), rows=rows) / B
            v /= np.linalg.norm(v)
        Av = self.forward(v, rows=rows)
        return float(np.vdot(Av, Av).real) / (B * float(np.vdot(v, v).real))

    def spgm_lipschitz(self, perm, pairs_per_batch, v0, iters: int) -> float:
        """Largest minibatch constant L_B over the minibatches of one epoch with permutation perm."""
        perm = np.asarray(perm)
        return max(self.power_iteration(v0, iters, pairs=perm[c:c + pairs_per_batch])
                   for c in range(0, perm.size, pairs_per_batch))

    def frobenius_bound(self) -> float:
        """||A||_F^2 / M, an upper bound on L = lambda_max(A^H A)/M (the trace bounds the largest
        eigenvalue of a positive semidefinite matrix).

        From Eq. 2, |A_mn|^2 = |p(f_m)|^2 / ((4 pi)^2 dT^2 dR^2), so the sum over the rows of one
        voxel factors into (sum_k |p_k|^2)(sum_t 1/dT^2)(sum_r 1/dR^2) / (4 pi)^2.
        """
        pos = self.geom.grid.positions()
        inv_t = np.zeros(self.N)
        for a in self._tx:
            inv_t += 1.0 / np.sum((pos - a) ** 2, axis=1)
        inv_r = np.zeros(self.N)
        for a in self._rx:
            inv_r += 1.0 / np.sum((pos - a) ** 2, axis=1)
        pk = float(self.K) if self._p is None else float(np.sum(self._p ** 2))
        return pk * float(np.sum(inv_t * inv_r)) / ((4.0 * math.pi) ** 2 * self.M)

    def minimiser_dense(self, y, lam, L, iters: int = 10000):
        """A minimiser of Eq. 3 (D + lambda R) for a problem small enough to hold A as a dense matrix:
        accelerated proximal gradient (FISTA: the Eq. 5 step from an extrapolated point, momentum
        (t_k - 1)/t_{k+1}, t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2) with step 1/L for `iters` iterations.
        Not the paper's method: a reference solution that the tests certify by its optimality
        conditions.  Returns (s, kkt) with kkt the largest violation of the l1 optimality conditions
        divided by lambda (w1 = 1, w2 = w3 = 0 only)."""
        assert self.w1 == 1.0 and self.w2 == 0.0 and self.w3 == 0.0
        A = self.dense(np.arange(self.M), self.all_cols())
        AH = A.conj().T
        y = np.asarray(y, dtype=np.complex128)
        eta = 1.0 / L
        s = np.zeros(self.N, dtype=np.complex128)
        z = s.copy()
        t = 1.0
        for _ in range(iters):
            s_new = prox_l1(z - eta * (AH @ (A @ z - y)) / self.M, eta * lam)
            t_new = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
            z = s_new + ((t - 1.0) / t_new) * (s_new - s)
            s, t = s_new, t_new
        g = AH @ (A @ s - y) / self.M
        nz = np.abs(s) > 0
        v_nz = float(np.max(np.abs(g[nz] + lam * s[nz] / np.abs(s[nz])))) if nz.any() else 0.0
        v_z = float(np.max(np.maximum(np.abs(g[~nz]) - lam, 0.0))) if (~nz).any() else 0.0
        return s, max(v_nz, v_z) / lam

    def lambda_max(self, y) -> float:
        """max_n |(A^H y)_n| / M: the smallest lambda for which s = 0 is a minimiser."""
        return float(np.max(np.abs(self.adjoint(y)))) / self.M


def prox_l1(z, alpha) -> np.ndarray:
    """prox of alpha * sum|.| on complex z: z * max(0, 1 - alpha/|z|), 0 if |z| <= alpha."""
    z = np.asarray(z, dtype=np.complex128)
    mag = np.abs(z)
    out = np.zeros_like(z)
    keep = mag > alpha
    out[keep] = z[keep] * (1.0 - alpha / mag[keep])
    return out


def voxel_groups(grid) -> np.ndarray:
    """Group index of every voxel (x fastest): the 2 x 2 x 1 blocks (ix // 2, iy // 2, iz); blocks at
    an odd grid edge hold fewer voxels."""
    ix = np.arange(grid.nx)
    iy = np.arange(grid.ny)
    iz = np.arange(grid.nz)
    gx, gy = (grid.nx + 1) // 2, (grid.ny + 1) // 2
    g = (iz[:, None, None] * gy + (iy // 2)[None, :, None]) * gx + (ix // 2)[None, None, :]
    return g.reshape(-1)


def group_norms(z, groups) -> np.ndarray:
    """||z_g||_2 of every group g (index = group id)."""
    z = np.asarray(z, dtype=np.complex128)
    return np.sqrt(np.bincount(groups, weights=np.abs(z) ** 2))


def prox_group(z, groups, alpha) -> np.ndarray:
    """prox of alpha * sum_g ||z_g||_2: z_g * max(0, 1 - alpha/||z_g||), 0 if ||z_g|| <= alpha."""
    z = np.asarray(z, dtype=np.complex128)
    nrm = group_norms(z, groups)
    scale = np.zeros_like(nrm)
    keep = nrm > alpha
    scale[keep] = 1.0 - alpha / nrm[keep]
    return z * scale[groups]


def nmse(a, b) -> float:
    """||a - b||^2 / ||b||^2."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.vdot(a - b, a - b).real / np.vdot(b, b).real)


def psnr_magnitude(a, ref) -> float:
    """PSNR over max-normalised reflectivity magnitudes against a reference (Sec. V)."""
    ma = np.abs(a) / max(np.max(np.abs(a)), 1e-300)
    mr = np.abs(ref) / max(np.max(np.abs(ref)), 1e-300)
    mse = float(np.mean((ma - mr) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)
