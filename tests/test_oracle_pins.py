"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test ties one part of the oracle to something the paper or mathematics
fixes: hand-derived values of Eq. 2 on right-triangle geometries, invariants
(adjoint identity, reciprocity, linear phase in frequency), brute force
against a dense matrix, a library eigensolver, optimality (KKT) conditions of
the l1 problem, and hand-worked prox values.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import Oracle, prox_l1
from paper_2509_00774_gb300 import inputs as I
from paper_2509_00774_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _one_voxel_geom(tx, rx, freqs, voxel=(0.0, 0.0, 0.4), pulse=None):
    grid = I.Grid(voxel[0], voxel[1], voxel[2], 0.01, 0.01, 0.01, 1, 1, 1)
    return I.Geometry(np.atleast_2d(np.asarray(tx, float)), np.atleast_2d(np.asarray(rx, float)),
                      np.asarray(freqs, float), grid, pulse=pulse)


def _tiny_random_geom(seed=0, T=3, R=2, K=5, grid=(4, 3, 2), pulse=False):
    rng = np.random.default_rng(seed)
    tx = np.concatenate([rng.uniform(-0.1, 0.1, (T, 2)), np.zeros((T, 1))], 1)
    rx = np.concatenate([rng.uniform(-0.1, 0.1, (R, 2)), np.zeros((R, 1))], 1)
    g = I.Grid(-0.02, -0.03, 0.3, 0.007, 0.011, 0.013, *grid)
    p = None
    if pulse:
        p = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    return I.Geometry(tx, rx, I.uniform_freqs(70e9, 80e9, K), g, pulse=p)


# ---------------------------------------------------------------------------
# Eq. 2: matrix element
# ---------------------------------------------------------------------------
def test_element_hand_cases():
    with open(os.path.join(GOLDEN, "eq2_hand_cases.json")) as f:
        gold = json.load(f)
    c = gold["c"]
    for case in gold["cases"]:
        geom = _one_voxel_geom(case["tx"], case["rx"], [case["f_over_c"] * c], gold["voxel"])
        a = Oracle(geom).element(0, 0)
        want = complex(case["expected_re"], case["expected_im"]) / case["expected_scale_inv"]
        assert abs(a - want) <= 1e-12 * abs(want), (case["why"], a, want)


def test_element_pulse_spectrum_scales_linearly():
    """p(f_m) multiplies the element (Eq. 2)."""
    p = np.array([0.5 - 2.0j])
    g0 = _one_voxel_geom([0.3, 0, 0], [0, 0, 0], [72e9])
    g1 = _one_voxel_geom([0.3, 0, 0], [0, 0, 0], [72e9], pulse=p)
    a0, a1 = Oracle(g0).element(0, 0), Oracle(g1).element(0, 0)
    assert abs(a1 - p[0] * a0) <= 1e-15 * abs(a1)


def test_row_index_mapping():
    """Row m = (t*R + r)*K + k: |A_m| = 1/(4 pi d_t d_r) with hand-built distances."""
    d_tx = [0.5, 0.41]                       # TX at x = 0.3, x = 0.09 (voxel at z = 0.4)
    d_rx = [0.4, 0.5, 0.58]                  # RX at origin, y = 0.3, y = 0.42
    tx = [[0.3, 0, 0], [0.09, 0, 0]]
    rx = [[0, 0, 0], [0, 0.3, 0], [0, 0.42, 0]]
    freqs = [70e9, 75e9]
    o = Oracle(_one_voxel_geom(tx, rx, freqs))
    col = o.dense(np.arange(o.M), [0])[:, 0]
    for t in range(2):
        for r in range(3):
            for k in range(2):
                m = (t * 3 + r) * 2 + k
                want_mag = 1.0 / (4 * math.pi * d_tx[t] * d_rx[r])
                assert abs(abs(col[m]) - want_mag) <= 1e-12 * want_mag
                # phase: -2 pi f_k (d_t + d_r)/c, compared on the unit circle
                want = np.exp(-2j * math.pi * ((freqs[k] * (d_tx[t] + d_rx[r]) / I.C_LIGHT) % 1.0))
                assert abs(col[m] / abs(col[m]) - want) <= 1e-9


def test_phase_is_linear_in_frequency():
    """For a uniform frequency grid the ratio A(f_{k+1})/A(f_k) is one fixed phasor."""
    geom = _tiny_random_geom(1, T=2, R=2, K=9)
    o = Oracle(geom)
    A = o.dense(np.arange(o.M), np.arange(o.N))
    pos = geom.grid.positions()
    for pair in range(o.P):
        t, r = divmod(pair, o.R)
        D = np.linalg.norm(geom.tx[t] - pos, axis=1) + np.linalg.norm(geom.rx[r] - pos, axis=1)
        df = geom.freq[1] - geom.freq[0]
        step = np.exp(-2j * math.pi * ((df * D / I.C_LIGHT) % 1.0))
        blk = A[pair * o.K:(pair + 1) * o.K]
        ratio = blk[1:] / blk[:-1]
        assert np.max(np.abs(ratio - step[None, :])) < 1e-9


def test_reciprocity_tx_rx_swap():
    """Eq. 2 is symmetric in the TX and RX positions."""
    geom = _tiny_random_geom(2, T=3, R=2, K=4)
    swapped = I.Geometry(geom.rx, geom.tx, geom.freq, geom.grid)
    a, b = Oracle(geom), Oracle(swapped)
    Aa = a.dense(np.arange(a.M), np.arange(a.N)).reshape(3, 2, 4, -1)
    Ab = b.dense(np.arange(b.M), np.arange(b.N)).reshape(2, 3, 4, -1)
    assert np.max(np.abs(Aa - Ab.transpose(1, 0, 2, 3))) < 1e-15


# ---------------------------------------------------------------------------
# matrix-free forward / adjoint
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("pulse", [False, True])
def test_forward_adjoint_match_dense(pulse):
    geom = _tiny_random_geom(3, pulse=pulse)
    o = Oracle(geom)
    A = o.dense(np.arange(o.M), np.arange(o.N))
    s = I.complex_gaussian(o.N, 10)
    r = I.complex_gaussian(o.M, 11)
    y = o.forward(s)
    g = o.adjoint(r)
    assert np.linalg.norm(y - A @ s) <= 1e-13 * np.linalg.norm(y)
    assert np.linalg.norm(g - A.conj().T @ r) <= 1e-13 * np.linalg.norm(g)
    # row and column subsets
    rows = np.array([7, 1, 22, 3])
    cols = np.array([5, 0, 17])
    assert np.allclose(o.forward(s[cols], rows=rows, cols=cols), A[np.ix_(rows, cols)] @ s[cols], rtol=1e-13, atol=0)
    assert np.allclose(o.adjoint(r[rows], rows=rows, cols=cols), A[np.ix_(rows, cols)].conj().T @ r[rows],
                       rtol=1e-13, atol=0)


def test_adjoint_identity_small_workload():
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    s = I.complex_gaussian(o.N, 20)
    r = I.complex_gaussian(o.M, 21)
    lhs = np.vdot(r, o.forward(s))           # <A s, r> conj-linear in r
    rhs = np.vdot(o.adjoint(r), s)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_forward_thread_count_independent():
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    s = I.complex_gaussian(o.N, 22)
    n0 = oracle.get_threads()
    try:
        oracle.set_threads(1)
        y1 = o.forward(s)
        oracle.set_threads(max(2, n0))
        y2 = o.forward(s)
    finally:
        oracle.set_threads(n0)
    assert np.array_equal(y1, y2)


def test_sparse_forward_equals_full():
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    s = w.scene_vector()
    a, b = o.forward(s), o.forward_sparse(s)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(a)


# ---------------------------------------------------------------------------
# prox (Eq. 5)
# ---------------------------------------------------------------------------
def test_prox_hand_cases():
    with open(os.path.join(GOLDEN, "prox_hand_cases.json")) as f:
        gold = json.load(f)
    for c in gold["cases"]:
        z = np.array([complex(*c["z"])])
        out = prox_l1(z, c["alpha"])[0]
        assert out == complex(*c["out"]), c


# ---------------------------------------------------------------------------
# PGM / SPGM (Eq. 5, Eq. 6)
# ---------------------------------------------------------------------------
def _kkt_violation(A, M, y, s, lam):
    """Optimality of D + lam*||.||_1 with grad D = A^H (A s - y)/M computed from the dense A."""
    g = A.conj().T @ (A @ s - y) / M
    nz = np.abs(s) > 0
    v_nz = np.max(np.abs(g[nz] + lam * s[nz] / np.abs(s[nz]))) if nz.any() else 0.0
    v_z = np.max(np.maximum(np.abs(g[~nz]) - lam, 0.0)) if (~nz).any() else 0.0
    return max(v_nz, v_z) / lam


def test_pgm_monotone_and_kkt_fixed_point():
    # overdetermined tiny problem (M=256 rows, N=48 voxels): PGM converges linearly
    w = W.small_T4R4_K16_16x16x8()
    grid = I.Grid(-0.03, -0.03, 0.25, 0.02, 0.02, 0.02, 4, 4, 3)
    geom = I.Geometry(w.geom.tx, w.geom.rx, w.geom.freq, grid)
    o = Oracle(geom)
    A = o.dense(np.arange(o.M), np.arange(o.N))
    s_true = I.point_scene(grid, 5, 0)
    y = I.add_noise(A @ s_true, I.complex_gaussian(o.M, 1), 30.0)
    L = float(np.linalg.eigvalsh(A.conj().T @ A / o.M)[-1])
    lam = 0.05 * o.lambda_max(y)
    eta = 1.0 / L
    s = np.zeros(o.N, dtype=np.complex128)
    F = [o.objective(y, s, lam)]
    for _ in range(400):
        s = o.pgm_step(y, s, eta, lam)
        F.append(o.objective(y, s, lam))
    F = np.array(F)
    assert np.all(np.diff(F) <= 1e-12 * F[0]), "PGM objective must not increase with eta = 1/L"
    assert _kkt_violation(A, o.M, y, s, lam) < 1e-6


def test_elastic_net_prox_hand_case_and_kkt():
    """R = w1 ||s||_1 + (w2/2)||s||^2: prox is the soft threshold then 1/(1 + eta lambda w2);
    the PGM fixed point satisfies the KKT conditions with the dense-matrix gradient."""
    w = W.small_T4R4_K16_16x16x8()
    grid = I.Grid(-0.03, -0.03, 0.25, 0.02, 0.02, 0.02, 4, 4, 3)
    geom = I.Geometry(w.geom.tx, w.geom.rx, w.geom.freq, grid)
    o = Oracle(geom, w1=1.0, w2=0.4)
    z = np.array([3 + 4j, 0.5 + 0j])
    out = o.prox(z, 2.5)                  # threshold 2.5, scale 1/(1 + 2.5*0.4) = 1/2
    assert out[0] == 0.75 + 1j and out[1] == 0
    A = o.dense(np.arange(o.M), np.arange(o.N))
    y = I.add_noise(A @ I.point_scene(grid, 5, 0), I.complex_gaussian(o.M, 1), 30.0)
    L = float(np.linalg.eigvalsh(A.conj().T @ A / o.M)[-1])
    lam = 0.05 * o.lambda_max(y)
    s = np.zeros(o.N, dtype=np.complex128)
    F = [o.objective(y, s, lam)]
    for _ in range(1000):
        s = o.pgm_step(y, s, 1.0 / L, lam)
        F.append(o.objective(y, s, lam))
    assert np.all(np.diff(F) <= 1e-12 * F[0])
    g = A.conj().T @ (A @ s - y) / o.M
    nz = np.abs(s) > 0
    v_nz = np.max(np.abs(g[nz] + lam * (s[nz] / np.abs(s[nz]) + 0.4 * s[nz])))
    v_z = np.max(np.maximum(np.abs(g[~nz]) - lam, 0.0)) if (~nz).any() else 0.0
    assert max(v_nz, v_z) / lam < 1e-6
    # Tikhonov only (w1 = 0): the PGM fixed point solves (A^H A/M + lam w2 I) s = A^H y / M
    t = Oracle(geom, w1=0.0, w2=2.0)
    s = np.zeros(o.N, dtype=np.complex128)
    for _ in range(2000):
        s = t.pgm_step(y, s, 1.0 / L, lam)
    exact = np.linalg.solve(A.conj().T @ A / o.M + lam * 2.0 * np.eye(o.N), A.conj().T @ y / o.M)
    assert np.linalg.norm(s - exact) <= 1e-8 * np.linalg.norm(exact)


def test_lambda_max_gives_zero_solution():
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    y = I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, 1), 30.0)
    lmax = o.lambda_max(y)
    s0 = np.zeros(o.N, dtype=np.complex128)
    for eta in (0.3, 7.0):
        assert not np.any(o.pgm_step(y, s0, eta, lmax * (1 + 1e-9)))
        assert np.any(o.pgm_step(y, s0, eta, lmax * 0.99))


def test_minibatch_gradient_is_unbiased():
    """Mean of the Eq. 6 minibatch gradients over one epoch = full gradient when B_p | P."""
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    s = I.complex_gaussian(o.N, 30) * 0.1
    y = I.complex_gaussian(o.M, 31)
    perm = I.epoch_permutation(o.P, 5, 0)
    gs = [o.minibatch_gradient(y, s, perm[c:c + 4]) for c in range(0, o.P, 4)]
    full = o.full_gradient(y, s)
    assert np.linalg.norm(np.mean(gs, axis=0) - full) <= 1e-12 * np.linalg.norm(full)


def test_rows_gradient_all_rows_is_full_gradient():
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    s = I.complex_gaussian(o.N, 33) * 0.1
    y = I.complex_gaussian(o.M, 34)
    full = o.full_gradient(y, s)
    assert np.linalg.norm(o.rows_gradient(y, s, np.arange(o.M)) - full) <= 1e-13 * np.linalg.norm(full)
    # a Cartesian minibatch: rows (pair, k) for the chosen pairs and frequencies, against the dense matrix
    pairs, mask = I.cartesian_minibatch(o.T, o.R, o.K, 2, 3, 5, seed=1, it=0)
    rows = np.array([p * o.K + k for p in pairs for k in np.flatnonzero(mask)])
    A = o.dense(rows, np.arange(o.N))
    want = A.conj().T @ (A @ s - y[rows]) / rows.size
    assert np.linalg.norm(o.rows_gradient(y, s, rows) - want) <= 1e-12 * np.linalg.norm(want)


def test_spgm_epoch_equals_sequence_of_steps():
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    y = I.complex_gaussian(o.M, 32)
    perm = I.epoch_permutation(o.P, 2, 0)
    s = np.zeros(o.N, dtype=np.complex128)
    a = o.spgm_epoch(y, s, perm, 5, 0.5, 0.001)   # 16 pairs in chunks 5,5,5,1
    b = s
    for c in (perm[0:5], perm[5:10], perm[10:15], perm[15:16]):
        rows = o.rows_of_pairs(c)
        A = o.dense(rows, np.arange(o.N))
        g = A.conj().T @ (A @ b - y[rows]) / rows.size
        b = prox_l1(b - 0.5 * g, 0.001 * 0.5)
    assert np.linalg.norm(a - b) <= 1e-12 * max(np.linalg.norm(b), 1e-30)


# ---------------------------------------------------------------------------
# power iteration vs a library eigensolver
# ---------------------------------------------------------------------------
def test_power_iteration_matches_eigvalsh():
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    A = o.dense(np.arange(o.M), np.arange(o.N))
    lam_top = float(np.linalg.eigvalsh(A @ A.conj().T / o.M)[-1])   # same nonzero spectrum as A^H A/M
    v0 = I.complex_gaussian(o.N, 3)
    # The top two eigenvalues are within 2.3% of each other here, so 50
    # iterations (the solver setting) leave a gap of a few percent; the
    # Rayleigh quotient is a lower bound and converges to the top eigenvalue.
    L50 = o.power_iteration(v0, 50)
    assert lam_top * 0.95 <= L50 <= lam_top * (1 + 1e-12)
    L500 = o.power_iteration(v0, 500)
    assert abs(L500 - lam_top) <= 1e-8 * lam_top


@pytest.mark.parametrize("pulse", [False, True])
def test_frobenius_bound_is_the_dense_trace(pulse):
    """||A||_F^2 / M from its closed form equals the sum of |A_mn|^2 over the dense matrix, and
    bounds the top eigenvalue of A^H A / M from above."""
    o = Oracle(_tiny_random_geom(4, T=3, R=4, K=6, grid=(5, 4, 3), pulse=pulse))
    A = o.dense(np.arange(o.M), np.arange(o.N))
    fro = float(np.sum(np.abs(A) ** 2)) / o.M
    assert abs(o.frobenius_bound() - fro) <= 1e-12 * fro
    lam_top = float(np.linalg.eigvalsh(A.conj().T @ A / o.M)[-1])
    assert lam_top <= o.frobenius_bound() * (1 + 1e-12)


# ---------------------------------------------------------------------------
# metrics
# ---------------------------------------------------------------------------
def test_psnr_and_nmse_closed_forms():
    ref = np.array([1.0, 0.5, 0.0, 0.25])
    a = np.array([1.0, 0.5, 0.1, 0.25])          # one magnitude off by 0.1 -> mse = 0.01/4
    assert abs(oracle.psnr_magnitude(a, ref) - 10 * math.log10(400.0)) < 1e-12
    assert abs(oracle.nmse(a, ref) - 0.01 / (1 + 0.25 + 0.0625)) < 1e-15


def test_group_prox_hand_case_and_groups():
    """2 x 2 x 1 voxel groups on a 3 x 2 x 1 grid (an odd edge group of two voxels): the group shrink
    scales a group by 1 - alpha/||z_g|| or zeroes it, exactly in FP64 for power-of-two factors."""
    from oracle import group_norms, prox_group, voxel_groups
    grid = I.Grid(0.0, 0.0, 0.3, 0.01, 0.01, 0.01, 3, 2, 1)
    g = voxel_groups(grid)
    assert list(g) == [0, 0, 1, 0, 0, 1]
    z = np.array([3, 0, 1j, 4j, 0, 0], dtype=np.complex128)
    assert np.allclose(group_norms(z, g), [5.0, 1.0])
    out = prox_group(z, g, 2.5)
    assert np.array_equal(out, np.array([1.5, 0, 0, 2j, 0, 0]))


def test_sparse_group_prox_minimises_its_definition():
    """prox(z) = argmin_p 1/2||p - z||^2 + a1 ||p||_1 + a2 sum_g ||p_g|| + (b/2)||p||^2: the oracle's
    closed form (soft threshold, group shrink, 1/(1 + b)) must not be beaten by any perturbation,
    including ones that zero single entries or whole groups (convex: a local minimum is global)."""
    w = W.small_T4R4_K16_16x16x8()
    grid = I.Grid(0.0, 0.0, 0.3, 0.01, 0.01, 0.01, 3, 4, 2)
    geom = I.Geometry(w.geom.tx, w.geom.rx, w.geom.freq, grid)
    from oracle import voxel_groups
    groups = voxel_groups(grid)
    rng = np.random.default_rng(5)
    seen_zero = seen_nonzero = False
    for a1, a2, b in ((0.3, 0.8, 0.0), (0.0, 1.5, 0.25), (0.7, 0.2, 0.5), (1.2, 2.5, 0.0)):
        o = Oracle(geom, w1=a1, w2=b, w3=a2)                  # prox(z, 1) uses a1, a2, b as written
        z = rng.standard_normal(o.N) + 1j * rng.standard_normal(o.N)

        def f(p):
            nrm = np.sqrt(np.bincount(groups, weights=np.abs(p) ** 2))
            return (0.5 * np.sum(np.abs(p - z) ** 2) + a1 * np.sum(np.abs(p)) + a2 * np.sum(nrm)
                    + 0.5 * b * np.sum(np.abs(p) ** 2))

        p = o.prox(z, 1.0)
        f0 = f(p)
        for t in range(3000):
            q = p.copy()
            kind = t % 3
            if kind == 0:
                q += (rng.standard_normal(o.N) + 1j * rng.standard_normal(o.N)) * 10.0 ** rng.uniform(-6, -1)
            elif kind == 1:
                q[rng.integers(o.N)] = 0.0
                q += (rng.standard_normal(o.N) + 1j * rng.standard_normal(o.N)) * 1e-4
            else:
                q[groups == rng.integers(groups.max() + 1)] = 0.0
            assert f(q) >= f0 - 1e-12 * max(1.0, abs(f0))
        seen_zero |= bool(np.any(p == 0))
        seen_nonzero |= bool(np.any(p != 0))
    assert seen_zero and seen_nonzero                   # both kinds of entries are exercised


# ---------------------------------------------------------------------------
# Eq. 3 / Eq. 4: data fidelity and objective on a hand-derived operator
# ---------------------------------------------------------------------------
def _hand_objective_geom():
    """TX at (0, 0.3, 0), RX at (0, -0.3, 0); two voxels at (-0.24, 0, 0.32) and (0.24, 0, 0.32) (one
    2 x 2 x 1 block: ix = 0, 1).  Every antenna-voxel distance is sqrt(0.24^2 + 0.3^2 + 0.32^2) = 0.5, so
    dT + dR = 1 m and dT dR = 1/4.  Frequencies c/4 and c/2 put 1/4 and 1/2 turn on that path, so by
    Eq. 2 every column of A is (e^{-j pi/2}, e^{-j pi}) / (4 pi / 4) = (-j, -1) / pi."""
    c = I.C_LIGHT
    grid = I.Grid(-0.24, 0.0, 0.32, 0.48, 0.01, 0.01, 2, 1, 1)
    return I.Geometry(np.array([[0.0, 0.3, 0.0]]), np.array([[0.0, -0.3, 0.0]]),
                      np.array([c / 4.0, c / 2.0]), grid)


def test_hand_operator_columns():
    o = Oracle(_hand_objective_geom())
    A = o.dense(np.arange(o.M), np.arange(o.N))
    want = np.array([[-1j, -1j], [-1.0, -1.0]]) / math.pi
    assert np.max(np.abs(A - want)) <= 1e-15


def test_data_fidelity_and_objective_hand_values():
    """s = pi (1, 2j): A s = (-j (1 + 2j), -(1 + 2j)) = (2 - j, -1 - 2j).  With y = A s + (3 + 4j, 0) the
    residual norm is 25, so D = 25 / (2 M) = 25/4 (M = 2 rows).  R terms: sum |s_n| = 3 pi,
    ||s||^2 = 5 pi^2, the one block's norm = sqrt(5) pi.  A dropped 1/2 or 1/M, or any missing or
    mis-weighted lambda R term, changes the value."""
    geom = _hand_objective_geom()
    s = math.pi * np.array([1.0, 2j])
    y = np.array([5 + 3j, -1 - 2j])
    o = Oracle(geom)                                           # the paper's l1 (w1 = 1)
    assert abs(o.data_fidelity(y, s) - 6.25) <= 1e-13
    lam = 0.25
    assert abs(o.objective(y, s, lam) - (6.25 + lam * 3 * math.pi)) <= 1e-13
    # zero residual: D = 0 exactly (up to rounding of A s)
    assert o.data_fidelity(np.array([2 - 1j, -1 - 2j]), s) <= 1e-28
    w1, w2, w3 = 1.0, 0.5, 2.0
    oe = Oracle(geom, w1=w1, w2=w2, w3=w3)
    R = w1 * 3 * math.pi + 0.5 * w2 * 5 * math.pi ** 2 + w3 * math.sqrt(5.0) * math.pi
    assert abs(oe.regulariser(s) - R) <= 1e-13 * R
    assert abs(oe.objective(y, s, lam) - (6.25 + lam * R)) <= 1e-13 * (6.25 + lam * R)


def test_data_fidelity_gradient_by_central_differences():
    """D is quadratic, so the central difference along e_n (and j e_n) is exact up to rounding and
    equals Re (and Im) of the gradient A^H (A s - y) / M.  This ties the scale of D to the gradient
    that the KKT pins check."""
    o = Oracle(_tiny_random_geom(7, T=2, R=3, K=4, grid=(3, 2, 2)))
    rng = np.random.default_rng(11)
    s = rng.standard_normal(o.N) + 1j * rng.standard_normal(o.N)
    y = (rng.standard_normal(o.M) + 1j * rng.standard_normal(o.M)) * 0.01
    g = o.full_gradient(y, s)
    eps = 1e-3
    fd = np.zeros(o.N, dtype=np.complex128)
    for n in range(o.N):
        for unit, part in ((1.0, "re"), (1j, "im")):
            sp, sm = s.copy(), s.copy()
            sp[n] += eps * unit
            sm[n] -= eps * unit
            d = (o.data_fidelity(y, sp) - o.data_fidelity(y, sm)) / (2 * eps)
            fd[n] += d if part == "re" else 1j * d
    assert np.max(np.abs(fd - g)) <= 1e-7 * np.max(np.abs(g))


# ---------------------------------------------------------------------------
# Sec. IV-A: the step of the minibatch gradient
# ---------------------------------------------------------------------------
def test_minibatch_power_iteration_matches_eigvalsh():
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    v0 = I.complex_gaussian(o.N, 3)
    for pairs in ([5], [3, 12, 0, 7]):
        A = o.dense(o.rows_of_pairs(pairs), np.arange(o.N))
        top = float(np.linalg.eigvalsh(A @ A.conj().T / A.shape[0])[-1])
        assert abs(o.power_iteration(v0, 300, pairs=pairs) - top) <= 1e-8 * top
    # the full list of pairs is the full-batch L
    assert abs(o.power_iteration(v0, 20, pairs=np.arange(o.P)) - o.power_iteration(v0, 20)) <= 1e-12 * o.M


def test_spgm_step_needs_the_minibatch_constant():
    """On the small workload a 4-pair minibatch has L_B up to several times the full-batch L, so
    SPGM with eta = 1/L diverges (the iterate grows without bound), while eta = 1/max L_B over the
    epoch's minibatches keeps it bounded: the reading of the step used for SPGM."""
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    y = I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, w.seeds["noise"]), w.snr_db)
    v0 = I.complex_gaussian(o.N, w.seeds["power"])
    L = o.power_iteration(v0, 50)
    LB = o.spgm_lipschitz(I.epoch_permutation(o.P, w.seeds["perm"], 0), 4, v0, 50)
    assert LB > 2.0 * L
    lam = 0.05 * o.lambda_max(y)
    norms = {}
    for name, eta in (("1/L", 1.0 / L), ("1/L_B", 1.0 / LB)):
        s = np.zeros(o.N, dtype=np.complex128)
        for e in range(20):
            s = o.spgm_epoch(y, s, I.epoch_permutation(o.P, w.seeds["perm"], e), 4, eta, lam)
        norms[name] = np.linalg.norm(s)
    ref = np.linalg.norm(w.scene_vector())        # the scene that made y
    assert norms["1/L"] > 1e4 * ref            # diverged
    assert norms["1/L_B"] < 10.0 * ref         # bounded


def test_dense_minimiser_is_optimal():
    """The reference minimiser of Eq. 3 used to time convergence: KKT conditions hold (from the dense
    gradient, checked independently here) and no PGM iterate started from it lowers the objective."""
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    y = I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, w.seeds["noise"]), w.snr_db)
    L = o.power_iteration(I.complex_gaussian(o.N, w.seeds["power"]), 50)
    lam = 0.05 * o.lambda_max(y)
    s, kkt = o.minimiser_dense(y, lam, L, iters=6000)
    A = o.dense(np.arange(o.M), np.arange(o.N))
    assert kkt < 1e-4 and _kkt_violation(A, o.M, y, s, lam) < 1e-4
    F = o.objective(y, s, lam)
    t = s
    for _ in range(50):
        t = o.pgm_step(y, t, 1.0 / L, lam)
        assert o.objective(y, t, lam) >= F - 1e-9 * F


# ---------------------------------------------------------------------------
# Sec. II: explicit voxel positions
# ---------------------------------------------------------------------------
def test_point_set_hand_cases_and_grid_equivalence():
    """A one-point set reproduces the hand-derived Eq. 2 values, and a point set holding a grid's
    positions reproduces the grid's dense matrix exactly."""
    with open(os.path.join(GOLDEN, "eq2_hand_cases.json")) as f:
        gold = json.load(f)
    c = gold["c"]
    for case in gold["cases"]:
        geom = I.Geometry(np.atleast_2d(np.asarray(case["tx"], float)), np.atleast_2d(np.asarray(case["rx"], float)),
                          np.array([case["f_over_c"] * c]), I.PointSet(np.array([gold["voxel"]], float)))
        a = Oracle(geom).element(0, 0)
        want = complex(case["expected_re"], case["expected_im"]) / case["expected_scale_inv"]
        assert abs(a - want) <= 1e-12 * abs(want), case["why"]
    g = _tiny_random_geom(3, T=2, R=3, K=4, grid=(4, 3, 2))
    pts = I.Geometry(g.tx, g.rx, g.freq, I.PointSet(g.grid.positions()))
    A = Oracle(g).dense(np.arange(g.M), np.arange(g.N))
    B = Oracle(pts).dense(np.arange(g.M), np.arange(g.N))
    assert np.array_equal(A, B)
    # a permuted point set permutes the columns
    perm = np.random.default_rng(1).permutation(g.N)
    C = Oracle(I.Geometry(g.tx, g.rx, g.freq, I.PointSet(g.grid.positions()[perm]))).dense(np.arange(g.M),
                                                                                           np.arange(g.N))
    assert np.array_equal(C, A[:, perm])
