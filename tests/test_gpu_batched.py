"""Batched SPGM of several uneven scenes per epoch (one CUDA graph, a branch per scene)."""
import numpy as np
import pytest

from oracle import Oracle, nmse
from paper_2509_00774_gb300 import inputs as I
from paper_2509_00774_gb300 import workloads as W
from tests.gpu_helpers import NMSE_TOL, make_ctx, to_dev, to_host

pytestmark = pytest.mark.gpu


def _c64(z):
    return np.asarray(z, dtype=np.complex64).astype(np.complex128)


def _tiny_scene(T, R, K, n, seed):
    tx, rx = I.boundary_array(T, R, 0.2)
    grid = I.lateral_grid(0.06, n, 0.3, 0.03, max(2, n // 2))
    return I.Geometry(tx, rx, I.uniform_freqs(70e9, 80e9, K), grid)


def _setup(geoms, seeds):
    ctxs, ys = [], []
    for g, sd in zip(geoms, seeds):
        ctx = make_ctx(g)
        o = Oracle(g)
        y = _c64(I.add_noise(o.forward_sparse(I.point_scene(g.grid, 10, sd)), I.complex_gaussian(o.M, sd + 1), 25.0))
        ctxs.append(ctx)
        ys.append(y)
    return ctxs, ys


def test_batch_matches_per_scene_epochs_and_oracle():
    import torch
    from paper_2509_00774_gb300.nfmimo import Batch
    geoms = [_tiny_scene(4, 4, 16, 12, 0), _tiny_scene(6, 4, 37, 8, 1), _tiny_scene(4, 6, 24, 10, 2),
             W.small_T4R4_K16_16x16x8().geom]
    ctxs, ys = _setup(geoms, [10, 20, 30, 40])
    bps = [4, 5, 16, 3]
    etas = [0.02, 0.03, 0.025, 0.02]
    lams = [1e-3, 2e-3, 1e-3, 5e-4]
    y_d = [to_dev(y) for y in ys]
    s_b = [torch.zeros(g.N, dtype=torch.complex64, device="cuda") for g in geoms]
    s_q = [torch.zeros(g.N, dtype=torch.complex64, device="cuda") for g in geoms]
    s_o = [np.zeros(g.N, dtype=np.complex128) for g in geoms]
    perm_d = [torch.zeros(g.P, dtype=torch.int32, device="cuda") for g in geoms]
    batch = Batch(ctxs)
    for e in range(3):
        for i, g in enumerate(geoms):
            p = I.epoch_permutation(g.P, 5 + i, e)
            perm_d[i].copy_(torch.from_numpy(p))
            ctxs[i].spgm_epoch(y_d[i], s_q[i], perm_d[i], bps[i], etas[i], lams[i])
            s_o[i] = Oracle(g).spgm_epoch(ys[i], s_o[i], p, bps[i], etas[i], lams[i])
        batch.spgm_epoch(y_d, s_b, perm_d, bps, etas, lams)     # captured once, replayed
        torch.cuda.synchronize()
        for i in range(len(geoms)):
            assert torch.equal(s_b[i], s_q[i]), (e, i)
            assert nmse(to_host(s_b[i]), s_o[i]) <= NMSE_TOL, (e, i)
    # a changed parameter re-captures
    etas[1] = 0.01
    batch.spgm_epoch(y_d, s_b, perm_d, bps, etas, lams)
    ctxs[1].spgm_epoch(y_d[1], s_q[1], perm_d[1], bps[1], etas[1], lams[1])
    for i in range(len(geoms)):
        if i != 1:
            ctxs[i].spgm_epoch(y_d[i], s_q[i], perm_d[i], bps[i], etas[i], lams[i])
    torch.cuda.synchronize()
    for i in range(len(geoms)):
        assert torch.equal(s_b[i], s_q[i])
    batch.close()


def test_batch_of_uneven_scenes_from_the_48_scene_set():
    """Three scenes of the 48-scene uneven set (largest grid 96 x 96 x 48 possible): batch == per scene."""
    import torch
    from paper_2509_00774_gb300.nfmimo import Batch
    ws = [W.batched_scene(i) for i in (0, 1, 2)]
    ctxs = [make_ctx(w.geom) for w in ws]
    ys, ss, sq, perms = [], [], [], []
    for i, (w, c) in enumerate(zip(ws, ctxs)):
        g = w.geom
        all_p = to_dev(np.arange(g.P), "int32")
        y = c.forward(all_p, to_dev(w.scene_vector()))
        ys.append(y)
        ss.append(torch.zeros(g.N, dtype=torch.complex64, device="cuda"))
        sq.append(torch.zeros(g.N, dtype=torch.complex64, device="cuda"))
        perms.append(to_dev(I.epoch_permutation(g.P, 9, 0), "int32"))
    etas = [0.01] * 3
    lams = [1e-3] * 3
    batch = Batch(ctxs)
    batch.spgm_epoch(ys, ss, perms, [16] * 3, etas, lams)
    for i in range(3):
        ctxs[i].spgm_epoch(ys[i], sq[i], perms[i], 16, etas[i], lams[i])
    torch.cuda.synchronize()
    for i in range(3):
        assert torch.equal(ss[i], sq[i]), ws[i].name
    batch.close()


def test_batched48_sampled_operator_matches_oracle():
    """Every scene of the 48-scene uneven set (grids 32..96, 8..24 TX/RX, 32..96 freqs): the forward of a
    16-pair minibatch on 64 sampled rows (scene = the workload's reflectivity, so the oracle's forward is
    a sparse sum) and the adjoint of a random residual on 64 sampled voxels, against the oracle."""
    from tests.gpu_helpers import REL_L2, ELEM_FACTOR
    worst = 0.0
    for i in range(48):
        w = W.batched_scene(i)
        g = w.geom
        o = Oracle(g)
        ctx = make_ctx(g)
        rng = np.random.default_rng(500 + i)
        pairs = I.epoch_permutation(g.P, 3, i)[:16]
        rows = o.rows_of_pairs(pairs)
        s = w.scene_vector()
        y = to_host(ctx.forward(to_dev(pairs, "int32"), to_dev(s)))
        sel = np.sort(rng.choice(rows.size, 64, replace=False))
        want = o.forward_sparse(_c64(s), rows=rows[sel])
        err = y[sel] - want
        rel = np.linalg.norm(err) / np.linalg.norm(want)
        rms = np.linalg.norm(want) / np.sqrt(want.size)
        assert rel <= REL_L2 and np.max(np.abs(err)) <= ELEM_FACTOR * REL_L2 * rms, (w.name, "forward", rel)
        r = _c64(I.complex_gaussian(rows.size, 600 + i))
        gad = to_host(ctx.adjoint(to_dev(pairs, "int32"), to_dev(r)))
        cols = np.sort(rng.choice(g.N, 64, replace=False))
        want = o.adjoint(r, rows=rows, cols=cols)
        err = gad[cols] - want
        rel2 = np.linalg.norm(err) / np.linalg.norm(want)
        rms = np.linalg.norm(want) / np.sqrt(want.size)
        assert rel2 <= REL_L2 and np.max(np.abs(err)) <= ELEM_FACTOR * REL_L2 * rms, (w.name, "adjoint", rel2)
        worst = max(worst, rel, rel2)
        ctx.close()
    print(f"[parity] 48 uneven scenes, sampled rows and voxels: worst rel l2 {worst:.2e}")


def test_batched48_smallest_scenes_spgm_match_oracle():
    """The 4 smallest scenes of the 48-scene set (by M N) solved together by one batched graph per epoch:
    3 SPGM epochs against the oracle's epochs with the same permutations (step 1/L_F, L_F = ||A||_F^2/M,
    which bounds every minibatch constant)."""
    import torch
    from paper_2509_00774_gb300.nfmimo import Batch
    ws = sorted((W.batched_scene(i) for i in range(48)), key=lambda w: w.geom.M * w.geom.N)[:4]
    ctxs, ys, y_d, s_b, s_o, perm_d, etas, lams = [], [], [], [], [], [], [], []
    for i, w in enumerate(ws):
        g = w.geom
        o = Oracle(g)
        y = _c64(I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, w.seeds["noise"]),
                             w.snr_db))
        ctxs.append(make_ctx(g))
        ys.append(y)
        y_d.append(to_dev(y))
        s_b.append(torch.zeros(g.N, dtype=torch.complex64, device="cuda"))
        s_o.append(np.zeros(g.N, dtype=np.complex128))
        perm_d.append(torch.zeros(g.P, dtype=torch.int32, device="cuda"))
        etas.append(float(np.float32(1.0 / o.frobenius_bound())))
        lams.append(float(np.float32(0.05 * o.lambda_max(y))))
    bps = [w.pairs_per_batch for w in ws]
    batch = Batch(ctxs)
    for e in range(3):
        for i, w in enumerate(ws):
            p = I.epoch_permutation(w.geom.P, w.seeds["perm"], e)
            perm_d[i].copy_(torch.from_numpy(p.astype(np.int32)))
            s_o[i] = Oracle(w.geom).spgm_epoch(ys[i], s_o[i], p, bps[i], etas[i], lams[i])
        batch.spgm_epoch(y_d, s_b, perm_d, bps, etas, lams)
        torch.cuda.synchronize()
        for i, w in enumerate(ws):
            err = nmse(to_host(s_b[i]), s_o[i])
            assert err <= NMSE_TOL, (w.name, e, err)
    batch.close()


def test_fused_batch_matches_branch_batch_and_oracle():
    """The fused batch (one forward, one reduction and one adjoint launch per step index over every scene)
    against the graph of per-scene branches on uneven scenes (grids 8..16, K 16..37, 4 to 36 pairs, ragged
    minibatches), and against the oracle's epochs; then three scenes of the 48-scene set.  The per-scene
    adjoint runs over blocks of two tiles with its own expansion table while the fused adjoint runs over
    the tiles, so the two agree to the FP32 operator's tolerance (rel 1e-5), not bit for bit."""
    import torch
    from paper_2509_00774_gb300.nfmimo import Batch
    geoms = [_tiny_scene(4, 4, 16, 12, 0), _tiny_scene(6, 4, 37, 8, 1), _tiny_scene(4, 6, 24, 10, 2),
             W.small_T4R4_K16_16x16x8().geom, _tiny_scene(6, 6, 20, 16, 3)]
    ctxs_f, ys = _setup(geoms, [10, 20, 30, 40, 50])
    ctxs_b = [make_ctx(g) for g in geoms]
    bps = [4, 5, 16, 3, 7]
    etas = [0.02, 0.03, 0.025, 0.02, 0.01]
    lams = [1e-3, 2e-3, 1e-3, 5e-4, 1e-3]
    y_d = [to_dev(y) for y in ys]
    s_f = [torch.zeros(g.N, dtype=torch.complex64, device="cuda") for g in geoms]
    s_b = [torch.zeros(g.N, dtype=torch.complex64, device="cuda") for g in geoms]
    s_o = [np.zeros(g.N, dtype=np.complex128) for g in geoms]
    perm_d = [torch.zeros(g.P, dtype=torch.int32, device="cuda") for g in geoms]
    fused, branches = Batch(ctxs_f), Batch(ctxs_b)
    fused.set_mode("fused")
    for c in ctxs_b:                                 # the same operator in both
        c.set_algorithm("chebyshev")
    for c in ctxs_f:
        c.set_algorithm("chebyshev")
    for e in range(3):
        for i, g in enumerate(geoms):
            p = I.epoch_permutation(g.P, 5 + i, e)
            perm_d[i].copy_(torch.from_numpy(p))
            s_o[i] = Oracle(g).spgm_epoch(ys[i], s_o[i], p, bps[i], etas[i], lams[i])
        fused.spgm_epoch(y_d, s_f, perm_d, bps, etas, lams)
        branches.spgm_epoch(y_d, s_b, perm_d, bps, etas, lams)
        torch.cuda.synchronize()
        for i in range(len(geoms)):
            a, b = to_host(s_f[i]), to_host(s_b[i])
            assert np.linalg.norm(a - b) <= 1e-5 * max(np.linalg.norm(b), 1e-30), (e, i)
            assert nmse(a, s_o[i]) <= NMSE_TOL, (e, i)
    fused.close()
    branches.close()
    # three scenes of the uneven set, fused against branches over one epoch
    ws = [W.batched_scene(i) for i in (0, 1, 2)]
    cf, cb = [make_ctx(w.geom) for w in ws], [make_ctx(w.geom) for w in ws]
    yy, sf, sb, pp = [], [], [], []
    for w, c in zip(ws, cf):
        g = w.geom
        yy.append(c.forward(to_dev(np.arange(g.P), "int32"), to_dev(w.scene_vector())))
        sf.append(torch.zeros(g.N, dtype=torch.complex64, device="cuda"))
        sb.append(torch.zeros(g.N, dtype=torch.complex64, device="cuda"))
        pp.append(to_dev(I.epoch_permutation(g.P, 9, 0), "int32"))
    for c in cf + cb:
        c.set_algorithm("chebyshev")
    bf, bb = Batch(cf), Batch(cb)
    bf.set_mode("fused")
    bf.spgm_epoch(yy, sf, pp, [16] * 3, [0.005] * 3, [1e-3] * 3)
    bb.spgm_epoch(yy, sb, pp, [16] * 3, [0.005] * 3, [1e-3] * 3)
    torch.cuda.synchronize()
    for i in range(3):
        a, b = to_host(sf[i]), to_host(sb[i])
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b), ws[i].name
    bf.close()
    bb.close()
