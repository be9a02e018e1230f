"""GPU SPGM (Eq. 5 with the Eq. 6 minibatch gradient), power iteration, objective and
lambda_max against the FP64 oracle, with identical seeded permutations."""
import numpy as np
import pytest

from oracle import Oracle, nmse
from paper_2509_00774_gb300 import inputs as I
from paper_2509_00774_gb300 import workloads as W
from paper_2509_00774_gb300.nfmimo import NfmError
from tests.gpu_helpers import NMSE_TOL, OBJ_TOL, make_ctx, spgm_eta, spgm_eta_epochs, to_dev, to_host

pytestmark = pytest.mark.gpu


def _c64(z):
    return np.asarray(z, dtype=np.complex64).astype(np.complex128)


def _small_problem():
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    y = _c64(I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, w.seeds["noise"]), w.snr_db))
    return w, o, y


def test_power_iteration_and_lambda_small():
    w, o, y = _small_problem()
    ctx = make_ctx(w.geom)
    v0 = _c64(I.complex_gaussian(o.N, w.seeds["power"]))
    L_gpu = ctx.power_iteration(to_dev(v0), 50)
    L_orc = o.power_iteration(v0, 50)
    assert abs(L_gpu - L_orc) <= 1e-4 * L_orc, (L_gpu, L_orc)
    lm_gpu = ctx.lambda_max(to_dev(y))
    lm_orc = o.lambda_max(y)
    assert abs(lm_gpu - lm_orc) <= 1e-5 * lm_orc, (lm_gpu, lm_orc)


def test_minibatch_power_iteration_small():
    """L_B = lambda_max(A_B^H A_B)/B of a minibatch (the SPGM step bound) against the oracle."""
    w, o, y = _small_problem()
    ctx = make_ctx(w.geom)
    v0 = _c64(I.complex_gaussian(o.N, w.seeds["power"]))
    for pairs in ([5], [3, 12, 0, 7], list(range(16))):
        L_gpu = ctx.power_iteration_pairs(to_dev(np.array(pairs), "int32"), to_dev(v0), 50)
        L_orc = o.power_iteration(v0, 50, pairs=pairs)
        assert abs(L_gpu - L_orc) <= 1e-4 * L_orc, (pairs, L_gpu, L_orc)
    perm = I.epoch_permutation(o.P, w.seeds["perm"], 0)
    LB_gpu = ctx.spgm_lipschitz(to_dev(perm, "int32"), 4, to_dev(v0), 50)
    assert abs(LB_gpu - o.spgm_lipschitz(perm, 4, v0, 50)) <= 1e-4 * LB_gpu


def test_objective_small():
    w, o, y = _small_problem()
    ctx = make_ctx(w.geom)
    s = _c64(I.point_scene(w.geom.grid, 40, 9)) * 0.7
    lam = 0.01
    F_gpu = ctx.objective(to_dev(y), to_dev(s), lam)
    F_orc = o.objective(y, s, lam)
    assert abs(F_gpu - F_orc) <= 1e-5 * F_orc, (F_gpu, F_orc)


@pytest.mark.parametrize("bp", [4, 5])
def test_spgm_small_matches_oracle(bp):
    """All 30 epochs of the small workload; bp = 5 leaves a 1-pair last chunk."""
    w, o, y = _small_problem()
    ctx = make_ctx(w.geom)
    eta = spgm_eta_epochs(o, w.seeds["perm"], bp, w.epochs)
    lam = float(np.float32(0.05 * o.lambda_max(y)))
    s_orc = np.zeros(o.N, dtype=np.complex128)
    s_gpu = to_dev(np.zeros(o.N))
    y_dev = to_dev(y)
    worst = 0.0
    for e in range(w.epochs):
        perm = I.epoch_permutation(o.P, w.seeds["perm"], e)
        s_orc = o.spgm_epoch(y, s_orc, perm, bp, eta, lam)
        ctx.spgm_epoch(y_dev, s_gpu, to_dev(perm, "int32"), bp, eta, lam)
        err = nmse(to_host(s_gpu), s_orc)
        worst = max(worst, err)
        assert err <= NMSE_TOL, f"epoch {e}: NMSE {err:.3e}"
    F_gpu = o.objective(y, to_host(s_gpu), lam)
    F_orc = o.objective(y, s_orc, lam)
    assert abs(F_gpu - F_orc) <= OBJ_TOL * F_orc


def test_pgm_matches_oracle():
    """Full-batch PGM (Eq. 5), 40 iterations on the small workload."""
    w, o, y = _small_problem()
    ctx = make_ctx(w.geom)
    L = o.power_iteration(I.complex_gaussian(o.N, w.seeds["power"]), 50)
    eta = float(np.float32(1.0 / L))
    lam = float(np.float32(0.05 * o.lambda_max(y)))
    s_orc = np.zeros(o.N, dtype=np.complex128)
    s_gpu = to_dev(np.zeros(o.N))
    y_dev = to_dev(y)
    for it in range(40):
        s_orc = o.pgm_step(y, s_orc, eta, lam)
        ctx.pgm_step(y_dev, s_gpu, eta, lam)
    assert nmse(to_host(s_gpu), s_orc) <= NMSE_TOL
    F_gpu = o.objective(y, to_host(s_gpu), lam)
    F_orc = o.objective(y, s_orc, lam)
    assert abs(F_gpu - F_orc) <= OBJ_TOL * F_orc


def test_solve_termination_rule():
    """Sec. V: epochs run until the change in reflectivity magnitudes drops below tol."""
    w, o, y = _small_problem()
    ctx = make_ctx(w.geom)
    eta = spgm_eta_epochs(o, w.seeds["perm"], 4, 60)
    lam = float(np.float32(0.05 * o.lambda_max(y)))
    tol, E = 2e-3, 60
    perms = np.stack([I.epoch_permutation(o.P, w.seeds["perm"], e) for e in range(E)]).astype(np.int32)
    # oracle: the same rule in FP64
    s = np.zeros(o.N, dtype=np.complex128)
    changes = []
    for e in range(E):
        s_new = o.spgm_epoch(y, s, perms[e], 4, eta, lam)
        changes.append(float(np.max(np.abs(np.abs(s_new) - np.abs(s)))))
        s = s_new
        if changes[-1] < tol:
            break
    s_gpu = to_dev(np.zeros(o.N))
    n_run, last = ctx.solve(to_dev(y), s_gpu, to_dev(perms, "int32"), 4, eta, lam, tol)
    assert last < tol or n_run == E
    # FP32 vs FP64 may cross the threshold one epoch apart
    assert abs(n_run - len(changes)) <= 1, (n_run, len(changes))
    assert abs(last - changes[n_run - 1]) <= 1e-3 * max(changes[n_run - 1], 1e-3) + 2e-5
    ref = o.spgm_epoch(y, np.zeros(o.N), perms[0], 4, eta, lam)
    for e in range(1, n_run):
        ref = o.spgm_epoch(y, ref, perms[e], 4, eta, lam)
    assert nmse(to_host(s_gpu), ref) <= NMSE_TOL


@pytest.mark.parametrize("comp", [(4, 2, 3), (16, 4, 4), (1, 1, 1)])
def test_cartesian_minibatch_steps_match_oracle(comp):
    """Minibatches of composition (#f, #Tx, #Rx) (Sec. IV-A) on the small workload."""
    n_f, n_t, n_r = comp
    w, o, y = _small_problem()
    ctx = make_ctx(w.geom)
    draws = [I.cartesian_minibatch(o.T, o.R, o.K, n_t, n_r, n_f, seed=4, it=it) for it in range(12)]
    eta = spgm_eta(o, [np.array([p * o.K + k for p in pairs for k in np.flatnonzero(mask)]) for pairs, mask in draws])
    lam = float(np.float32(0.05 * o.lambda_max(y)))
    s_orc = np.zeros(o.N, dtype=np.complex128)
    s_gpu = to_dev(np.zeros(o.N))
    y_dev = to_dev(y)
    import torch
    for it in range(12):
        pairs, mask = I.cartesian_minibatch(o.T, o.R, o.K, n_t, n_r, n_f, seed=4, it=it)
        rows = np.array([p * o.K + k for p in pairs for k in np.flatnonzero(mask)])
        s_orc = o.spgm_step_rows(y, s_orc, rows, eta, lam)
        ctx.spgm_step_freqs(y_dev, s_gpu, to_dev(pairs, "int32"), torch.from_numpy(mask).cuda(), eta, lam)
        assert nmse(to_host(s_gpu), s_orc) <= NMSE_TOL, it


@pytest.mark.parametrize("w1,w2", [(1.0, 0.5), (0.0, 3.0)])
def test_elastic_net_and_tikhonov_spgm_match_oracle(w1, w2):
    """Other regularisers (Sec. III): R = w1 ||s||_1 + (w2/2)||s||^2, 10 epochs on the small workload."""
    w, _, y = _small_problem()
    o = Oracle(w.geom, w1=w1, w2=w2)
    ctx = make_ctx(w.geom)
    ctx.set_regularizer(w1, w2)
    eta = spgm_eta_epochs(o, w.seeds["perm"], 4, 10)
    lam = float(np.float32(0.05 * o.lambda_max(y)))
    s_orc = np.zeros(o.N, dtype=np.complex128)
    s_gpu = to_dev(np.zeros(o.N))
    y_dev = to_dev(y)
    for e in range(10):
        perm = I.epoch_permutation(o.P, w.seeds["perm"], e)
        s_orc = o.spgm_epoch(y, s_orc, perm, 4, eta, lam)
        ctx.spgm_epoch(y_dev, s_gpu, to_dev(perm, "int32"), 4, eta, lam)
        assert nmse(to_host(s_gpu), s_orc) <= NMSE_TOL, e
    F_gpu = ctx.objective(y_dev, s_gpu, lam)
    F_orc = o.objective(y, to_host(s_gpu), lam)
    assert abs(F_gpu - F_orc) <= 1e-5 * F_orc


def test_spgm_host_buffers_match_device():
    w, o, y = _small_problem()
    ctx = make_ctx(w.geom)
    eta, lam = 0.01, 1e-4
    perms = np.stack([I.epoch_permutation(o.P, 2, e) for e in range(3)]).astype(np.int32)
    s_dev = to_dev(np.zeros(o.N))
    y_dev = to_dev(y)
    for e in range(3):
        ctx.spgm_epoch(y_dev, s_dev, to_dev(perms[e], "int32"), 4, eta, lam)
    s_host = np.zeros(o.N, dtype=np.complex64)
    ctx.spgm_epochs_host(y.astype(np.complex64), s_host, perms, 4, eta, lam)
    assert np.array_equal(s_host, s_dev.cpu().numpy())


def test_spgm_mid_three_epochs():
    """Mid workload (N = 131072, 16 pairs x 64 frequencies per minibatch): the first three SPGM
    epochs in full, every iterate of the first epoch and the end of each epoch against the oracle.
    The step is 1/||A||_F^2 * M (the oracle's closed-form bound on L; a power iteration on this
    size is too slow for the oracle) and lambda = 0.05 max|A^H y|/M from the oracle."""
    w = W.mid_T16R16_K64_64x64x32()
    o = Oracle(w.geom)
    y = _c64(I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, w.seeds["noise"]), w.snr_db))
    ctx = make_ctx(w.geom)
    eta = float(np.float32(1.0 / o.frobenius_bound()))
    lam = float(np.float32(0.05 * o.lambda_max(y)))
    s_orc = np.zeros(o.N, dtype=np.complex128)
    s_gpu = to_dev(np.zeros(o.N))
    y_dev = to_dev(y)
    bp = w.pairs_per_batch
    for e in range(3):
        perm = I.epoch_permutation(o.P, w.seeds["perm"], e)
        if e == 0:
            for c in range(o.P // bp):
                pairs = perm[bp * c:bp * (c + 1)]
                s_orc = o.spgm_step(y, s_orc, pairs, eta, lam)
                ctx.spgm_step(y_dev, s_gpu, to_dev(pairs, "int32"), eta, lam)
                err = nmse(to_host(s_gpu), s_orc)
                assert err <= NMSE_TOL, f"step {c}: NMSE {err:.3e}"
        else:
            s_orc = o.spgm_epoch(y, s_orc, perm, bp, eta, lam)
            ctx.spgm_epoch(y_dev, s_gpu, to_dev(perm, "int32"), bp, eta, lam)
        err = nmse(to_host(s_gpu), s_orc)
        print(f"[parity] mid SPGM epoch {e}: NMSE {err:.3e}")
        assert err <= NMSE_TOL, f"epoch {e}: NMSE {err:.3e}"
    assert np.count_nonzero(s_orc) > 0


def test_power_iteration_mid_matches_oracle_rayleigh_quotient():
    """Mid workload: L from nfm_power_iteration (50 iterations) against the oracle's FP64 Rayleigh
    quotient ||A v||^2 / (M ||v||^2) at the iterate v_50 of the same iteration run through the GPU
    forward and adjoint (one full oracle application instead of 50), and the Rayleigh quotient at
    v_50 bounds the one at v_0 from above (the iteration climbs towards the top eigenvalue)."""
    import torch
    w = W.mid_T16R16_K64_64x64x32()
    o = Oracle(w.geom)
    ctx = make_ctx(w.geom)
    v0 = _c64(I.complex_gaussian(o.N, w.seeds["power"]))
    L_gpu = ctx.power_iteration(to_dev(v0), 50)
    pairs = to_dev(np.arange(o.P), "int32")
    v = to_dev(v0)
    for _ in range(50):
        u = ctx.adjoint(pairs, ctx.forward(pairs, v))
        v = u / torch.linalg.vector_norm(u)
    v50 = to_host(v)

    def rayleigh(x):
        ax = o.forward(x)
        return float(np.vdot(ax, ax).real) / (o.M * float(np.vdot(x, x).real))

    rq50 = rayleigh(v50)
    print(f"[parity] mid power iteration: L_gpu {L_gpu:.6f}, oracle Rayleigh quotient at v_50 {rq50:.6f}")
    assert abs(L_gpu - rq50) <= 1e-4 * rq50, (L_gpu, rq50)
    assert rq50 >= rayleigh(v0)


# ---------------------------------------------------------------------------
# errors
# ---------------------------------------------------------------------------
def test_out_of_range_pair_is_reported():
    w, o, y = _small_problem()
    ctx = make_ctx(w.geom)
    s = to_dev(np.zeros(o.N))
    ctx.forward(to_dev(np.array([0, 16]), "int32"), s)
    with pytest.raises(NfmError) as ei:
        ctx.synchronize()
    assert ei.value.code == -1
    ctx.synchronize()    # flag cleared


def test_invalid_geometry_rejected():
    from paper_2509_00774_gb300.nfmimo import Context
    w = W.small_T4R4_K16_16x16x8()
    g = w.geom
    ctx = Context(0)
    bad_freq = I.Geometry(g.tx, g.rx, np.array([72e9, -73e9, 75e9]), g.grid)
    too_many = I.Geometry(g.tx, g.rx, I.uniform_freqs(70e9, 80e9, 129), g.grid)
    inside = I.Geometry(np.array([[0.0, 0.0, 0.27]]), g.rx, g.freq, g.grid)
    for bad in (bad_freq, too_many, inside):
        with pytest.raises(NfmError) as ei:
            ctx.set_geometry(bad)
        assert ei.value.code == -1
    with pytest.raises(NfmError) as ei:
        ctx.forward(to_dev(np.array([0]), "int32"), to_dev(np.zeros(g.N)), to_dev(np.zeros(g.K)))
    assert ei.value.code == -4          # no geometry yet
    ctx.set_geometry(g)
    with pytest.raises(NfmError):
        ctx.spgm_step(to_dev(np.zeros(g.M)), to_dev(np.zeros(g.N)), to_dev(np.array([0]), "int32"), -1.0, 0.1)


def test_empty_minibatch_rejected():
    """A minibatch of zero pairs is an argument error for every operator entry point (host check,
    nothing is launched); the context stays usable."""
    w, o, y = _small_problem()
    ctx = make_ctx(w.geom)
    empty = to_dev(np.array([], dtype=np.int32), "int32")
    s = to_dev(np.zeros(o.N))
    for call in (lambda: ctx.forward(empty, s, to_dev(np.zeros(1))),
                 lambda: ctx.adjoint(empty, to_dev(np.zeros(1)), to_dev(np.zeros(o.N))),
                 lambda: ctx.spgm_step(to_dev(y), s, empty, 1e-3, 1e-3)):
        with pytest.raises(NfmError) as ei:
            call()
        assert ei.value.code == -1
    g = to_host(ctx.adjoint(to_dev(np.arange(16), "int32"), to_dev(np.zeros(o.M))))
    assert np.all(g == 0)


@pytest.mark.parametrize("grid_kind,w1,w2,w3,precision", [("small", 1.0, 0.0, 1.0, "fp32"),
                                                          ("odd", 0.5, 0.5, 2.0, "fp32"),
                                                          ("odd", 1.0, 0.0, 1.0, "tc_bf16x3")])
def test_group_regulariser_spgm_matches_oracle(grid_kind, w1, w2, w3, precision):
    """R = w1 ||s||_1 + (w2/2)||s||^2 + w3 sum_g ||s_g||_2 over 2 x 2 x 1 voxel blocks (the prox is the
    soft threshold, the block shrink, the w2 scaling): 10 SPGM epochs against the oracle, on the small
    grid and on a 15 x 13 x 5 grid whose edge blocks hold fewer voxels; then the FP64 objective."""
    w = W.small_T4R4_K16_16x16x8()
    if grid_kind == "small":
        geom = w.geom
    else:
        g0 = w.geom.grid
        grid = I.Grid(g0.x0, g0.y0, g0.z0, g0.dx, g0.dy, g0.dz, 15, 13, 5)
        geom = I.Geometry(w.geom.tx, w.geom.rx, w.geom.freq, grid)
    o = Oracle(geom, w1=w1, w2=w2, w3=w3)
    y = I.add_noise(o.forward_sparse(I.point_scene(geom.grid, 12, 3)), I.complex_gaussian(o.M, 4), 25.0)
    y = y.astype(np.complex64).astype(np.complex128)
    ctx = make_ctx(geom, algorithm="chebyshev")
    ctx.set_precision(precision)
    ctx.set_regularizer(w1, w2)
    ctx.set_group_weight(w3)
    eta = spgm_eta_epochs(o, 6, 4, 10)
    lam = float(np.float32(0.2 * o.lambda_max(y)))     # strong enough that 20-35% of the blocks vanish
    s_orc = np.zeros(o.N, dtype=np.complex128)
    s_gpu = to_dev(np.zeros(o.N))
    y_dev = to_dev(y)
    for e in range(10):
        perm = I.epoch_permutation(o.P, 6, e)
        s_orc = o.spgm_epoch(y, s_orc, perm, 4, eta, lam)
        ctx.spgm_epoch(y_dev, s_gpu, to_dev(perm, "int32"), 4, eta, lam)
        assert nmse(to_host(s_gpu), s_orc) <= NMSE_TOL, e
    from oracle import group_norms, voxel_groups
    zero_groups = np.sum(group_norms(s_orc, voxel_groups(geom.grid)) == 0)
    print(f"[parity] group regulariser {grid_kind} {precision}: NMSE {nmse(to_host(s_gpu), s_orc):.2e}, "
          f"{zero_groups} zero blocks")
    assert 0 < zero_groups < voxel_groups(geom.grid).max() + 1
    F_gpu = ctx.objective(y_dev, s_gpu, lam)
    F_orc = o.objective(y, to_host(s_gpu), lam)
    assert abs(F_gpu - F_orc) <= 1e-5 * F_orc


def test_group_regulariser_needs_the_expansion_operator():
    from paper_2509_00774_gb300.nfmimo import NfmError
    w = W.small_T4R4_K16_16x16x8()
    ctx = make_ctx(w.geom, algorithm="direct")
    ctx.set_group_weight(1.0)
    y = to_dev(np.zeros(w.geom.M))
    s = to_dev(np.zeros(w.geom.N))
    with pytest.raises(NfmError):
        ctx.spgm_epoch(y, s, to_dev(I.epoch_permutation(w.geom.P, 0, 0), "int32"), 4, 0.01, 0.01)
    with pytest.raises(NfmError):
        ctx.set_group_weight(-1.0)


def test_bounds_checked_build_matches_and_reports():
    """The bounds-checked build (-DNFM_BOUNDS_CHECK) gives the normal build's results on the default
    operator path (to FP32 rounding: the extra checks change where the compiler contracts a multiply and an
    add into one FMA, so the two builds need not agree bit for bit), and when the test hook halves the extents its kernels receive, a checked access past the
    declared extent (still inside the real buffer) raises the device flag and the next synchronise reports
    NFM_ERR_STATE; the context stays usable."""
    from paper_2509_00774_gb300 import build as nb
    from paper_2509_00774_gb300.nfmimo import Context
    w, o, y = _small_problem()
    path = nb.build(check=True)
    ref = make_ctx(w.geom, "chebyshev")
    chk = Context(0, library=path)
    chk.set_geometry(w.geom)
    chk.set_algorithm("chebyshev")
    pairs = to_dev(I.epoch_permutation(o.P, 4, 0)[:5], "int32")
    s0 = _c64(I.complex_gaussian(o.N, 12)) * 0.1
    y_d = to_dev(y)
    outs = []
    for ctx in (ref, chk):
        s = to_dev(s0)
        for _ in range(3):
            ctx.spgm_step(y_d, s, pairs, 0.003, 1e-3)
        ctx.synchronize()
        outs.append(to_host(s))
    rel = np.linalg.norm(outs[1] - outs[0]) / np.linalg.norm(outs[0])
    print(f"[check build] 3 SPGM steps vs the normal build: rel_l2 {rel:.2e}")
    assert rel <= 1e-6
    chk.set_test_hooks(chk.HOOK_SHRINK_EXTENTS)
    s = to_dev(s0)
    chk.spgm_step(y_d, s, pairs, 0.003, 1e-3)
    with pytest.raises(NfmError) as ei:
        chk.synchronize()
    assert ei.value.code == -4 and "bounds" in str(ei.value)
    chk.set_test_hooks(0)
    chk.spgm_step(y_d, s, pairs, 0.003, 1e-3)
    chk.synchronize()
    ref.set_test_hooks(ref.HOOK_SHRINK_EXTENTS)    # the normal build ignores the extents
    ref.spgm_step(y_d, to_dev(s0), pairs, 0.003, 1e-3)
    ref.synchronize()
    ref.close()
    chk.close()
