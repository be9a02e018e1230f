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
