"""Python binding of the nfmimo C-ABI (include/nfmimo.h): argument marshalling only.

Every entry point of the C library has a method of the same name on
`Context`.  Device vectors are torch tensors on the context's GPU
(complex64 for complex vectors, int32 for pair lists); host vectors for the
`*_host` call are numpy arrays or CPU tensors.  All compute runs in the CUDA
library; there is no fallback: if the library is missing or no GPU is
present the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnfmimo.so")

NFM_OK = 0
_STATUS = {-1: "NFM_ERR_ARG", -2: "NFM_ERR_CUDA", -3: "NFM_ERR_NOMEM", -4: "NFM_ERR_STATE",
           -5: "NFM_ERR_TIMEOUT", -6: "NFM_ERR_NUMERIC"}

_lib = None
_libs = {}


class NfmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


def load_library(path: str | None = None):
    """Load libnfmimo.so, or the library at `path` (e.g. the bounds-checked libnfmimo_check.so); raises if it
    has not been built.  Each path is loaded once."""
    global _lib
    path = path or LIB_PATH
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2509_00774_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i, f, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double
    sig = {
        "nfm_create": (i, [ctypes.POINTER(vp), i, vp]),
        "nfm_destroy": (None, [vp]),
        "nfm_last_error": (ctypes.c_char_p, [vp]),
        "nfm_set_stream": (i, [vp, vp]),
        "nfm_set_geometry": (i, [vp, vp, i, vp, i, vp, i, vp, ctypes.POINTER(_Grid), d]),
        "nfm_set_geometry_points": (i, [vp, vp, i, vp, i, vp, i, vp, vp, ctypes.c_longlong, d]),
        "nfm_set_precision": (i, [vp, i]),
        "nfm_set_algorithm": (i, [vp, i]),
        "nfm_algorithm_info": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(d)]),
        "nfm_expansion_info": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "nfm_cheb_coefficients": (i, [d, d, i, i, vp]),
        "nfm_set_forward_shape": (i, [vp, i, i, i, i, i, i]),
        "nfm_set_group_weight": (i, [vp, d]),
        "nfm_autotune": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                             ctypes.POINTER(i)]),
        "nfm_set_regularizer": (i, [vp, d, d]),
        "nfm_dims": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                         ctypes.POINTER(ctypes.c_longlong)]),
        "nfm_forward": (i, [vp, vp, i, vp, vp]),
        "nfm_forward_noalloc": (i, [vp, vp, i, vp, vp]),
        "nfm_adjoint": (i, [vp, vp, i, vp, vp]),
        "nfm_residual": (i, [vp, vp, i, vp, vp, vp]),
        "nfm_spgm_step": (i, [vp, vp, vp, vp, i, f, f]),
        "nfm_spgm_epoch": (i, [vp, vp, vp, vp, i, f, f]),
        "nfm_spgm_epochs_host": (i, [vp, vp, vp, vp, i, i, f, f]),
        "nfm_pgm_step": (i, [vp, vp, vp, f, f]),
        "nfm_spgm_step_freqs": (i, [vp, vp, vp, vp, i, vp, i, f, f]),
        "nfm_solve": (i, [vp, vp, vp, vp, i, i, f, f, d, ctypes.POINTER(i), ctypes.POINTER(d)]),
        "nfm_prox_step": (i, [vp, vp, vp, f, f, f, ctypes.c_longlong, vp]),
        "nfm_prox_step_backward": (i, [vp, vp, vp, f, f, f, ctypes.c_longlong, vp, vp, vp, vp]),
        "nfm_prox_group_step": (i, [vp, vp, vp, f, f, f, f, vp]),
        "nfm_prox_group_step_backward": (i, [vp, vp, vp, f, f, f, f, vp, vp, vp, vp]),
        "nfm_power_iteration": (i, [vp, i, vp, ctypes.POINTER(d)]),
        "nfm_power_iteration_pairs": (i, [vp, vp, i, i, vp, ctypes.POINTER(d)]),
        "nfm_objective": (i, [vp, vp, vp, d, ctypes.POINTER(d)]),
        "nfm_lambda_max": (i, [vp, vp, ctypes.POINTER(d)]),
        "nfm_synchronize": (i, [vp]),
        "nfm_set_test_hooks": (i, [vp, i, i]),
        "nfm_profile_enable": (i, [vp, i]),
        "nfm_batch_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(vp), i, vp]),
        "nfm_batch_destroy": (None, [vp]),
        "nfm_batch_spgm_epoch": (i, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(i), ctypes.POINTER(f), ctypes.POINTER(f)]),
        "nfm_batch_last_error": (ctypes.c_char_p, [vp]),
        "nfm_batch_set_mode": (i, [vp, i]),
        "nfm_profile_report": (i, [vp, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong), i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _libs[path] = L
    if path == LIB_PATH:
        _lib = L
    return L


def cheb_coefficients(z_step: float, K: int, L: int, k_center: float = 0.0):
    """FP64 table b[k, l] = b_l((k - k_center) z_step) of exp(-j z t) = sum_l (-j)^l b_l(z) T_l(t)
    (host only)."""
    import numpy as np
    out = np.zeros((int(K), int(L)), dtype=np.float64)
    rc = load_library().nfm_cheb_coefficients(float(z_step), float(k_center), int(K), int(L),
                                              out.ctypes.data_as(ctypes.c_void_p))
    if rc != NFM_OK:
        raise NfmError(rc, "nfm_cheb_coefficients: invalid arguments")
    return out


def _ptr(t, dtype, name, device=None):
    """Data pointer of a contiguous torch tensor of the given dtype (complex64 -> float pairs)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device is not None:
        if t.device.type != "cuda" or t.device.index != device:
            raise ValueError(f"{name} must live on cuda:{device}, got {t.device}")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One nfm_ctx: a geometry on one GPU and a stream."""

    def __init__(self, device: int = 0, stream=None, library: str | None = None):
        """library: path of an alternative build of the library (the bounds-checked one); default libnfmimo.so."""
        import torch
        self._lib = load_library(library)
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self._stream = stream
        h = ctypes.c_void_p()
        rc = self._lib.nfm_create(ctypes.byref(h), self.device, ctypes.c_void_p(stream.cuda_stream))
        if rc != NFM_OK:
            raise NfmError(rc, self._lib.nfm_last_error(None).decode())
        self._h = h
        self.T = self.R = self.K = self.N = None

    def _check(self, rc):
        if rc != NFM_OK:
            raise NfmError(rc, self._lib.nfm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nfm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # ---------------------------------------------------------------------
    def set_stream(self, stream):
        self._stream = stream
        self._check(self._lib.nfm_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))

    def set_geometry(self, geom):
        """geom: an `inputs.Geometry` (FP64 antennas, frequencies, grid, pulse, c)."""
        tx = np.ascontiguousarray(geom.tx, dtype=np.float64)
        rx = np.ascontiguousarray(geom.rx, dtype=np.float64)
        fr = np.ascontiguousarray(geom.freq, dtype=np.float64)
        pulse = None
        if geom.pulse is not None:
            p = np.asarray(geom.pulse, dtype=np.complex128)
            pulse = np.ascontiguousarray(np.stack([p.real, p.imag], 1))
        g = geom.grid
        vp = ctypes.c_void_p
        pp = None if pulse is None else pulse.ctypes.data_as(vp)
        if hasattr(g, "xyz"):                 # explicit voxel positions (an inputs.PointSet)
            xyz = np.ascontiguousarray(g.xyz, dtype=np.float64)
            self._check(self._lib.nfm_set_geometry_points(
                self._h, tx.ctypes.data_as(vp), tx.shape[0], rx.ctypes.data_as(vp), rx.shape[0],
                fr.ctypes.data_as(vp), fr.shape[0], pp, xyz.ctypes.data_as(vp), xyz.shape[0], float(geom.c)))
        else:
            grid = _Grid(g.x0, g.y0, g.z0, g.dx, g.dy, g.dz, g.nx, g.ny, g.nz)
            self._check(self._lib.nfm_set_geometry(
                self._h, tx.ctypes.data_as(vp), tx.shape[0], rx.ctypes.data_as(vp), rx.shape[0],
                fr.ctypes.data_as(vp), fr.shape[0], pp, ctypes.byref(grid), float(geom.c)))
        self.T, self.R, self.K, self.N = tx.shape[0], rx.shape[0], fr.shape[0], g.N
        self.P = self.T * self.R
        self.M = self.P * self.K

    def set_geometry_points(self, geom):
        """set_geometry for a geometry whose voxels are an explicit point set (inputs.PointSet)."""
        if not hasattr(geom.grid, "xyz"):
            raise ValueError("set_geometry_points needs a geometry whose grid is an inputs.PointSet")
        self.set_geometry(geom)

    PRECISION = {"fp32": 0, "tc_bf16x3": 1, "tc_fp16x3": 2}

    def set_precision(self, mode):
        """Adjoint arithmetic: "fp32" (CUDA cores), "tc_bf16x3" or "tc_fp16x3" (tensor cores)."""
        self._check(self._lib.nfm_set_precision(self._h, self.PRECISION[mode] if isinstance(mode, str) else int(mode)))

    ALGORITHM = {"auto": 0, "direct": 1, "chebyshev": 2}

    def set_algorithm(self, algo):
        """Frequency evaluation of the FP32 operator: "auto", "direct" or "chebyshev"."""
        self._check(self._lib.nfm_set_algorithm(self._h, self.ALGORITHM[algo] if isinstance(algo, str) else int(algo)))

    def algorithm_info(self):
        """(algorithm in use: "direct" | "chebyshev", expansion length L, z of the highest frequency)."""
        a, n, z = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(self._lib.nfm_algorithm_info(self._h, ctypes.byref(a), ctypes.byref(n), ctypes.byref(z)))
        return {1: "direct", 2: "chebyshev"}[a.value], n.value, z.value

    def expansion_info(self):
        """(expansion length, voxels per block) of the FP32 expansion operator (forward and adjoint): blocks
        of two tiles (256 voxels) on a regular grid, the 128-voxel tiles otherwise."""
        n, v = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.nfm_expansion_info(self._h, ctypes.byref(n), ctypes.byref(v)))
        return n.value, v.value

    cheb_coefficients = staticmethod(cheb_coefficients)

    def autotune(self, n_pairs):
        """Time the expansion forward's launch shapes (and, with algorithm "auto", the expansion
        against the direct recurrence) for n_pairs-pair minibatches and keep the fastest; returns
        {"algorithm", "threads", "lanes_per_group", "pairs_per_cta", "chunks"}."""
        a, t, g, p, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.nfm_autotune(self._h, int(n_pairs), ctypes.byref(a), ctypes.byref(t), ctypes.byref(g),
                                           ctypes.byref(p), ctypes.byref(c)))
        return {"algorithm": {1: "direct", 2: "chebyshev"}[a.value], "threads": t.value, "lanes_per_group": g.value,
                "pairs_per_cta": p.value, "chunks": c.value}

    def set_forward_shape(self, n_pairs, shape):
        """Apply a forward launch shape for n_pairs-pair minibatches without timing (e.g. a dict that
        autotune returned earlier: "algorithm", "threads", "lanes_per_group", "pairs_per_cta", "chunks")."""
        algo = {"chebyshev": 2, "direct": 1}[shape.get("algorithm", "chebyshev")]
        self._check(self._lib.nfm_set_forward_shape(self._h, int(n_pairs), algo, int(shape["threads"]),
                                                    int(shape["lanes_per_group"]), int(shape["pairs_per_cta"]),
                                                    int(shape["chunks"])))

    def set_group_weight(self, w3=0.0):
        """Adds w3 sum_g ||s_g||_2 over 2 x 2 x 1 voxel blocks to R(s) (0 = off); needs the expansion operator."""
        self._check(self._lib.nfm_set_group_weight(self._h, float(w3)))

    def set_regularizer(self, w1=1.0, w2=0.0):
        """R(s) = w1 ||s||_1 + (w2/2) ||s||_2^2 for every SPGM/PGM step and the objective."""
        self._check(self._lib.nfm_set_regularizer(self._h, float(w1), float(w2)))

    def dims(self):
        T, R, K, N = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        self._check(self._lib.nfm_dims(self._h, ctypes.byref(T), ctypes.byref(R), ctypes.byref(K),
                                       ctypes.byref(N)))
        return T.value, R.value, K.value, N.value

    # ---------------------------------------------------------------------
    def _c(self, t, name):
        import torch
        return _ptr(t, torch.complex64, name, self.device)

    def _i(self, t, name):
        import torch
        return _ptr(t, torch.int32, name, self.device)

    def _need_geom(self):
        if self.K is None:
            raise NfmError(-4, "no geometry: call set_geometry first")

    def _sizes(self, **want):
        """Raise NfmError(-1) unless every named tensor has the given element count (checked before any
        raw pointer reaches the library, which cannot see the extents of what it is given)."""
        for name, (t, n) in want.items():
            if t.numel() != n:
                raise NfmError(-1, f"{name} has {t.numel()} elements, expected {n}")

    def forward(self, pairs, s, y=None):
        """y = A_B s for the pair list `pairs` (int32, device); returns y [n_pairs*K]."""
        import torch
        self._need_geom()
        n = pairs.numel()
        if y is None:
            y = torch.empty(n * self.K, dtype=torch.complex64, device=s.device)
        self._sizes(s=(s, self.N), y=(y, n * self.K))
        self._check(self._lib.nfm_forward(self._h, self._i(pairs, "pairs"), n, self._c(s, "s"), self._c(y, "y")))
        return y

    def forward_noalloc(self, pairs, s, y):
        """y = A_B s through the allocation-free entry point (y must be given; nothing is allocated)."""
        self._need_geom()
        self._sizes(s=(s, self.N), y=(y, pairs.numel() * self.K))
        self._check(self._lib.nfm_forward_noalloc(self._h, self._i(pairs, "pairs"), pairs.numel(),
                                                  self._c(s, "s"), self._c(y, "y")))
        return y

    def residual(self, pairs, s, y, r=None):
        """r = A_B s - y_B for the pair list `pairs` (int32, device), y the full measurement vector [P*K];
        returns r [n_pairs*K]."""
        import torch
        self._need_geom()
        n = pairs.numel()
        if r is None:
            r = torch.empty(n * self.K, dtype=torch.complex64, device=s.device)
        self._sizes(s=(s, self.N), y=(y, self.P * self.K), r=(r, n * self.K))
        self._check(self._lib.nfm_residual(self._h, self._i(pairs, "pairs"), n, self._c(s, "s"), self._c(y, "y"),
                                           self._c(r, "r")))
        return r

    def adjoint(self, pairs, r, g=None):
        """g = A_B^H r; returns g [N]."""
        import torch
        self._need_geom()
        n = pairs.numel()
        if g is None:
            g = torch.empty(self.N, dtype=torch.complex64, device=r.device)
        self._sizes(r=(r, n * self.K), g=(g, self.N))
        self._check(self._lib.nfm_adjoint(self._h, self._i(pairs, "pairs"), n, self._c(r, "r"), self._c(g, "g")))
        return g

    def spgm_step(self, y, s, pairs, eta, lam):
        self._need_geom()
        self._sizes(y=(y, self.P * self.K), s=(s, self.N))
        self._check(self._lib.nfm_spgm_step(self._h, self._c(y, "y"), self._c(s, "s"), self._i(pairs, "pairs"),
                                            pairs.numel(), float(eta), float(lam)))
        return s

    def spgm_epoch(self, y, s, perm, pairs_per_batch, eta, lam):
        self._need_geom()
        self._sizes(y=(y, self.P * self.K), s=(s, self.N), perm=(perm, self.P))
        self._check(self._lib.nfm_spgm_epoch(self._h, self._c(y, "y"), self._c(s, "s"), self._i(perm, "perm"),
                                             int(pairs_per_batch), float(eta), float(lam)))
        return s

    def spgm_epochs_host(self, y_host, s_host, perms_host, pairs_per_batch, eta, lam):
        """Host-buffer SPGM: y_host [P*K] complex64, s_host [N] complex64 (updated in place),
        perms_host [n_epochs, P] int32 (numpy arrays or CPU tensors, ideally pinned)."""
        def hp(a, dt, name):
            if hasattr(a, "data_ptr"):
                if a.device.type != "cpu" or not a.is_contiguous():
                    raise ValueError(f"{name} must be a contiguous CPU tensor")
                return ctypes.c_void_p(a.data_ptr())
            a = np.asarray(a)
            if a.dtype != dt or not a.flags.c_contiguous:
                raise ValueError(f"{name} must be a contiguous {dt} array")
            return a.ctypes.data_as(ctypes.c_void_p)
        perms = perms_host
        n_epochs = perms.shape[0] if perms.ndim == 2 else 1
        self._check(self._lib.nfm_spgm_epochs_host(
            self._h, hp(y_host, np.complex64, "y_host"), hp(s_host, np.complex64, "s_host"),
            hp(perms, np.int32, "perms_host"), n_epochs, int(pairs_per_batch), float(eta), float(lam)))
        return s_host

    def spgm_step_freqs(self, y, s, pairs, freq_mask, eta, lam, n_freq=None):
        """SPGM step on the rows (pairs x selected frequencies); freq_mask: uint8 device tensor [K].
        n_freq (the number of set mask entries) is counted on the device when not given."""
        import torch
        if n_freq is None:
            n_freq = int(freq_mask.count_nonzero())
        self._check(self._lib.nfm_spgm_step_freqs(
            self._h, self._c(y, "y"), self._c(s, "s"), self._i(pairs, "pairs"), pairs.numel(),
            _ptr(freq_mask, torch.uint8, "freq_mask", self.device), n_freq, float(eta), float(lam)))
        return s

    def pgm_step(self, y, s, eta, lam):
        """One full-batch PGM iteration (every pair), s updated in place."""
        self._check(self._lib.nfm_pgm_step(self._h, self._c(y, "y"), self._c(s, "s"), float(eta), float(lam)))
        return s

    def solve(self, y, s, perms, pairs_per_batch, eta, lam, tol, max_epochs=None):
        """Epochs until the change in reflectivity magnitudes over an epoch < tol.
        perms: int32 device tensor [max_epochs, P].  Returns (epochs_run, last_change)."""
        n = perms.shape[0] if max_epochs is None else int(max_epochs)
        ep = ctypes.c_int()
        ch = ctypes.c_double()
        self._check(self._lib.nfm_solve(self._h, self._c(y, "y"), self._c(s, "s"), self._i(perms, "perms"), n,
                                        int(pairs_per_batch), float(eta), float(lam), float(tol),
                                        ctypes.byref(ep), ctypes.byref(ch)))
        return ep.value, ch.value

    def prox_step(self, s, g, step, alpha, out, shrink=1.0):
        """out = shrink prox_alpha(s - step g) (Eq. 5; shrink = 1/(1 + eta lambda w2) for the elastic net);
        out may be s."""
        self._check(self._lib.nfm_prox_step(self._h, self._c(s, "s"), self._c(g, "g"), float(step), float(alpha),
                                            float(shrink), s.numel(), self._c(out, "out")))
        return out

    def prox_step_backward(self, s, g, step, alpha, grad_out, grad_s, grad_g, scalars, shrink=1.0):
        """Backward of prox_step; scalars: float64 device tensor [3] <- (dL/dstep, dL/dalpha, dL/dshrink)."""
        import torch
        ps = self._c(grad_s, "grad_s") if grad_s is not None else None
        pg = self._c(grad_g, "grad_g") if grad_g is not None else None
        if scalars.numel() < 3:
            raise NfmError(-1, "scalars needs 3 float64 entries")
        self._check(self._lib.nfm_prox_step_backward(
            self._h, self._c(s, "s"), self._c(g, "g"), float(step), float(alpha), float(shrink), s.numel(),
            self._c(grad_out, "grad_out"), ps, pg, _ptr(scalars, torch.float64, "scalars", self.device)))

    def prox_group_step(self, s, g, step, alpha, alpha_g, out, shrink=1.0):
        """out = shrink G_{alpha_g}(prox_alpha(s - step g)), G the block shrink over the grid's 2 x 2 x 1 voxel
        blocks (the prox of the sparse-group regulariser, Eq. 5); s, g, out: [N]; out may be s."""
        self._need_geom()
        self._sizes(s=(s, self.N), g=(g, self.N), out=(out, self.N))
        self._check(self._lib.nfm_prox_group_step(self._h, self._c(s, "s"), self._c(g, "g"), float(step),
                                                  float(alpha), float(alpha_g), float(shrink), self._c(out, "out")))
        return out

    def prox_group_step_backward(self, s, g, step, alpha, alpha_g, grad_out, grad_s, grad_g, scalars, shrink=1.0):
        """Backward of prox_group_step; scalars: float64 device tensor [4] <- (dL/dstep, dL/dalpha,
        dL/dalpha_g, dL/dshrink)."""
        import torch
        self._need_geom()
        self._sizes(s=(s, self.N), g=(g, self.N), grad_out=(grad_out, self.N))
        for name, t in (("grad_s", grad_s), ("grad_g", grad_g)):
            if t is not None:
                self._sizes(**{name: (t, self.N)})
        ps = self._c(grad_s, "grad_s") if grad_s is not None else None
        pg = self._c(grad_g, "grad_g") if grad_g is not None else None
        if scalars.numel() < 4:
            raise NfmError(-1, "scalars needs 4 float64 entries")
        self._check(self._lib.nfm_prox_group_step_backward(
            self._h, self._c(s, "s"), self._c(g, "g"), float(step), float(alpha), float(alpha_g), float(shrink),
            self._c(grad_out, "grad_out"), ps, pg, _ptr(scalars, torch.float64, "scalars", self.device)))

    def power_iteration(self, v0, iters: int = 50) -> float:
        L = ctypes.c_double()
        self._check(self._lib.nfm_power_iteration(self._h, int(iters), self._c(v0, "v0"), ctypes.byref(L)))
        return L.value

    def power_iteration_pairs(self, pairs, v0, iters: int = 50) -> float:
        """L_B = lambda_max(A_B^H A_B) / B for the minibatch of the listed pairs (int32, device)."""
        self._need_geom()
        self._sizes(v0=(v0, self.N))
        L = ctypes.c_double()
        self._check(self._lib.nfm_power_iteration_pairs(self._h, self._i(pairs, "pairs"), pairs.numel(), int(iters),
                                                        self._c(v0, "v0"), ctypes.byref(L)))
        return L.value

    def spgm_lipschitz(self, perm, pairs_per_batch, v0, iters: int = 50) -> float:
        """Largest L_B over the minibatches that one epoch with permutation `perm` (int32, device) takes."""
        P = perm.numel()
        return max(self.power_iteration_pairs(perm[c:c + pairs_per_batch], v0, iters)
                   for c in range(0, P, int(pairs_per_batch)))

    def objective(self, y, s, lam) -> float:
        F = ctypes.c_double()
        self._check(self._lib.nfm_objective(self._h, self._c(y, "y"), self._c(s, "s"), float(lam), ctypes.byref(F)))
        return F.value

    def lambda_max(self, y) -> float:
        out = ctypes.c_double()
        self._check(self._lib.nfm_lambda_max(self._h, self._c(y, "y"), ctypes.byref(out)))
        return out.value

    def synchronize(self):
        self._check(self._lib.nfm_synchronize(self._h))

    HOOK_TC_SKIP_ISSUE = 1
    HOOK_SHRINK_EXTENTS = 2

    def set_test_hooks(self, flags=0, wait_ms=0):
        """Error-path hooks for tests: flags = HOOK_TC_SKIP_ISSUE makes the tensor-core kernels issue no
        MMA, so their bounded waits (wait_ms; 0 = 1000 ms) run out and the next synchronising call raises
        NfmError(-5) with the output left unwritten.  flags = 0 restores normal operation."""
        self._check(self._lib.nfm_set_test_hooks(self._h, int(flags), int(wait_ms)))

    PROFILE_KINDS = ("forward_partial", "forward_reduce", "adjoint", "reductions")

    def profile_enable(self, on: bool = True):
        self._check(self._lib.nfm_profile_enable(self._h, 1 if on else 0))

    def profile_report(self) -> dict:
        """{kind: (total_ms, launches)} since the last report (synchronises)."""
        n = len(self.PROFILE_KINDS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        self._check(self._lib.nfm_profile_report(self._h, ms, cnt, n))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.PROFILE_KINDS)}


class Batch:
    """nfm_batch: one SPGM epoch of many scenes (each a Context with its own geometry) per call,
    run as one CUDA graph with a concurrent branch per scene."""

    def __init__(self, contexts, stream=None):
        import torch
        self._lib = load_library()
        self.contexts = list(contexts)
        if stream is None:
            stream = torch.cuda.current_stream(self.contexts[0].device)
        self._stream = stream
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.handle.value for c in self.contexts])
        h = ctypes.c_void_p()
        rc = self._lib.nfm_batch_create(ctypes.byref(h), arr, len(self.contexts), ctypes.c_void_p(stream.cuda_stream))
        if rc != NFM_OK:
            raise NfmError(rc, self._lib.nfm_last_error(None).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nfm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    MODES = {"branches": 0, "fused": 1}

    def set_mode(self, mode):
        """"branches": a graph branch per scene (default); "fused": one launch per phase and step over all
        scenes (FP32 expansion operator, L <= 20)."""
        rc = self._lib.nfm_batch_set_mode(self._h, self.MODES[mode] if isinstance(mode, str) else int(mode))
        if rc != NFM_OK:
            raise NfmError(rc, self._lib.nfm_batch_last_error(self._h).decode())

    def spgm_epoch(self, ys, ss, perms, pairs_per_batch, etas, lams):
        """ys, ss, perms: per-scene device tensors (complex64, complex64 in/out, int32)."""
        import torch
        n = len(self.contexts)
        P = ctypes.c_void_p
        def ptrs(ts, dt, name):
            return (P * n)(*[_ptr(t, dt, name, self.contexts[0].device).value for t in ts])
        bp = (ctypes.c_int * n)(*[int(x) for x in pairs_per_batch])
        et = (ctypes.c_float * n)(*[float(x) for x in etas])
        la = (ctypes.c_float * n)(*[float(x) for x in lams])
        rc = self._lib.nfm_batch_spgm_epoch(self._h, ptrs(ys, torch.complex64, "y"), ptrs(ss, torch.complex64, "s"),
                                            ptrs(perms, torch.int32, "perm"), bp, et, la)
        if rc != NFM_OK:
            raise NfmError(rc, self._lib.nfm_batch_last_error(self._h).decode())
