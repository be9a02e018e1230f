"""Helpers for the GPU parity tests: move seeded inputs to the device, compare with the oracle.

Tolerances (FP32 path against the FP64 oracle):
  * REL_L2 = 1e-5: relative l2 error of an operator application (the FP32
    operator bound stated for this method's GPU form).
  * ELEM = 5 * REL_L2 * rms(reference): no single element may be off by more
    than five times the l2 budget spread evenly over the elements.  The
    per-element error is a sum of many independent FP32 rounding and phase
    errors, i.e. close to Gaussian, and 5 sigma is not reached by chance over
    the <= 1e5 elements a test compares.
  * Where the dense matrix is cheap (small cases) the reference size of output
    m is the root-sum-square of its terms, sqrt(sum_n |A_mn s_n|^2), instead
    of |y_m|.  The FP32 error of a sum scales with that quantity; it equals
    |y_m| in expectation for random-phase terms, but a short sum that happens
    to cancel (one pair, one frequency) would otherwise look ill-conditioned.
  * SPGM iterates: NMSE <= 1e-4 against the oracle's iterate after the same
    epochs with the same permutations; objective within 1e-3 relative.
"""
import numpy as np

REL_L2 = 1e-5
ELEM_FACTOR = 5.0
NMSE_TOL = 1e-4
OBJ_TOL = 1e-3


def torch_mod():
    import torch
    return torch


def to_dev(z, dtype="complex64"):
    torch = torch_mod()
    a = np.ascontiguousarray(np.asarray(z))
    if dtype == "complex64":
        return torch.from_numpy(a.astype(np.complex64)).cuda()
    return torch.from_numpy(a.astype(np.int32)).cuda()


def to_host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def assert_close_operator(got, want, what="", scale=None):
    """scale: optional per-element root-sum-square of the terms (FP64)."""
    got = np.asarray(got)
    want = np.asarray(want)
    assert got.shape == want.shape, (got.shape, want.shape)
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    err = got - want
    ref = np.asarray(scale) if scale is not None else np.abs(want)
    rel = np.linalg.norm(err) / np.linalg.norm(ref)
    rms = np.linalg.norm(ref) / np.sqrt(ref.size)
    worst = np.max(np.abs(err)) / rms
    print(f"[parity] {what}: n={err.size} rel_l2={rel:.2e} worst/rms={worst:.2e}")
    assert rel <= REL_L2, f"{what}: relative l2 error {rel:.3e} > {REL_L2:.0e}"
    assert worst <= ELEM_FACTOR * REL_L2, f"{what}: worst element error {worst:.3e} rms > {ELEM_FACTOR * REL_L2:.0e}"
    return rel, worst


# operator algorithm for make_ctx ("auto" unless a test module parametrizes it)
ALGORITHM = "auto"


def make_ctx(geom, algorithm=None):
    from paper_2509_00774_gb300.nfmimo import Context
    ctx = Context(0)
    ctx.set_geometry(geom)
    algo = algorithm or ALGORITHM
    ctx.set_algorithm(algo)
    if algo != "auto":
        assert ctx.algorithm_info()[0] == algo
    return ctx


def term_scale(dense_block, x):
    """sqrt(sum_j |B_ij x_j|^2) for every row i of an FP64 dense block."""
    return np.sqrt((np.abs(dense_block) ** 2) @ (np.abs(x) ** 2))


def spgm_eta(o, row_sets):
    """SPGM step for a small problem: 1 / max over the minibatches of L_B = lambda_max(A_B A_B^H) / B from
    the oracle's dense rows (FP64 eigensolver), rounded to FP32.  A step of 1/L (full batch) makes SPGM
    diverge on these geometries: a few pairs' L_B is several times L."""
    cols = np.arange(o.N)
    LB = max(float(np.linalg.eigvalsh((lambda A: A @ A.conj().T / A.shape[0])(o.dense(np.asarray(r), cols)))[-1])
             for r in row_sets)
    return float(np.float32(1.0 / LB))


def spgm_eta_epochs(o, seed, bp, epochs):
    """spgm_eta over every minibatch of `epochs` epochs of seeded permutations in chunks of bp pairs."""
    from paper_2509_00774_gb300 import inputs as I
    sets = []
    for e in range(epochs):
        perm = I.epoch_permutation(o.P, seed, e)
        sets += [o.rows_of_pairs(perm[c:c + bp]) for c in range(0, o.P, bp)]
    uniq = {tuple(sorted(r)) for r in sets}
    return spgm_eta(o, [np.array(r) for r in uniq])
