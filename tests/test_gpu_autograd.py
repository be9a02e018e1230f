"""Differentiation through the CUDA operators (autograd.Function wrappers, unrolled SPGM),
checked against the FP64 oracle: oracle gradients and FP64 central finite differences."""
import numpy as np
import pytest

from oracle import Oracle, prox_l1
from paper_2509_00774_gb300 import inputs as I
from paper_2509_00774_gb300 import workloads as W
from tests.gpu_helpers import make_ctx, to_dev, to_host

pytestmark = pytest.mark.gpu


def _c64(z):
    return np.asarray(z, dtype=np.complex64).astype(np.complex128)


def test_forward_op_gradient_matches_oracle_and_fd():
    """L(s) = ||A_B s - y||^2: grad = 2 A_B^H (A_B s - y) (dL/dRe + j dL/dIm)."""
    import torch
    from paper_2509_00774_gb300.autograd import forward_op
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    ctx = make_ctx(w.geom)
    pairs = np.array([3, 12, 0, 7])
    rows = o.rows_of_pairs(pairs)
    s = _c64(I.complex_gaussian(o.N, 40)) * 0.3
    y = _c64(I.complex_gaussian(rows.size, 41))
    s_d = to_dev(s).requires_grad_(True)
    L = (forward_op(ctx, to_dev(pairs, "int32"), s_d) - to_dev(y)).abs().pow(2).sum()
    L.backward()
    got = to_host(s_d.grad)
    want = 2.0 * o.adjoint(o.forward(s, rows=rows) - y, rows=rows)
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)
    # FP64 central differences on a few coordinates, through the oracle
    h = 1e-6
    loss = lambda v: float(np.sum(np.abs(o.forward(v, rows=rows) - y) ** 2))
    for j in (0, 777, 2047):
        e = np.zeros(o.N, dtype=np.complex128)
        e[j] = h
        d_re = (loss(s + e) - loss(s - e)) / (2 * h)
        d_im = (loss(s + 1j * e) - loss(s - 1j * e)) / (2 * h)
        assert abs(got[j] - (d_re + 1j * d_im)) <= 1e-4 * abs(d_re + 1j * d_im) + 1e-6


def test_residual_op_value_and_gradient_match_oracle():
    """r = A_B s - y_B fused in one launch (y the full measurement vector): value against the oracle's rows,
    and the gradient of ||r||^2, 2 A_B^H (A_B s - y_B)."""
    from paper_2509_00774_gb300.autograd import residual_op
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    ctx = make_ctx(w.geom)
    pairs = np.array([9, 2, 15, 4, 4])
    rows = o.rows_of_pairs(pairs)
    s = _c64(I.complex_gaussian(o.N, 44)) * 0.3
    y = _c64(I.complex_gaussian(o.M, 45))
    s_d = to_dev(s).requires_grad_(True)
    r = residual_op(ctx, to_dev(pairs, "int32"), s_d, to_dev(y))
    want_r = o.forward(s, rows=rows) - y[rows]
    assert np.linalg.norm(to_host(r) - want_r) <= 1e-5 * np.linalg.norm(want_r)
    r.abs().pow(2).sum().backward()
    want = 2.0 * o.adjoint(want_r, rows=rows)
    assert np.linalg.norm(to_host(s_d.grad) - want) <= 1e-5 * np.linalg.norm(want)


def test_adjoint_op_gradient_matches_oracle():
    """L(r) = ||A_B^H r - t||^2: grad = 2 A_B (A_B^H r - t)."""
    from paper_2509_00774_gb300.autograd import adjoint_op
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    ctx = make_ctx(w.geom)
    pairs = np.array([1, 9, 14])
    rows = o.rows_of_pairs(pairs)
    r = _c64(I.complex_gaussian(rows.size, 42))
    t = _c64(I.complex_gaussian(o.N, 43)) * 0.01
    r_d = to_dev(r).requires_grad_(True)
    L = (adjoint_op(ctx, to_dev(pairs, "int32"), r_d) - to_dev(t)).abs().pow(2).sum()
    L.backward()
    got = to_host(r_d.grad)
    want = 2.0 * o.forward(o.adjoint(r, rows=rows) - t, rows=rows)
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


def test_prox_step_backward_matches_fd():
    """out = prox_alpha(s - step g); L = sum Re(conj(c) out).  FP64 central differences of the
    oracle prox for grad_s, grad_g, dL/dstep and dL/dalpha (entries near |z| = alpha excluded)."""
    import torch
    from paper_2509_00774_gb300.autograd import prox_step
    w = W.small_T4R4_K16_16x16x8()
    ctx = make_ctx(w.geom)
    n = 4000
    rng = np.random.default_rng(44)
    s = _c64(I.complex_gaussian(n, 45))
    g = _c64(I.complex_gaussian(n, 46))
    c = _c64(I.complex_gaussian(n, 47))
    step, alpha = 0.3, 0.6
    z = s - step * g
    keep = np.abs(np.abs(z) - alpha) > 1e-2           # away from the kink of the prox
    s_d = to_dev(s).requires_grad_(True)
    g_d = to_dev(g).requires_grad_(True)
    st = torch.tensor(step, dtype=torch.float64, requires_grad=True)
    al = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    out = prox_step(ctx, s_d, g_d, st, al)
    L = (torch.conj(to_dev(c)) * out).real.sum()
    L.backward()
    gs, gg = to_host(s_d.grad), to_host(g_d.grad)

    def loss(s_, g_, st_, al_):
        return float(np.sum((np.conj(c) * prox_l1(s_ - st_ * g_, al_)).real[keep]))

    h = 1e-6
    idx = np.flatnonzero(keep)[:: max(1, keep.sum() // 40)]
    for j in idx:
        e = np.zeros(n, dtype=np.complex128)
        e[j] = h
        fd_s = (loss(s + e, g, step, alpha) - loss(s - e, g, step, alpha)) / (2 * h) + \
            1j * (loss(s + 1j * e, g, step, alpha) - loss(s - 1j * e, g, step, alpha)) / (2 * h)
        assert abs(gs[j] - fd_s) <= 1e-4 * max(1.0, abs(fd_s)), (j, gs[j], fd_s)
        assert abs(gg[j] + step * fd_s) <= 1e-4 * max(1.0, abs(fd_s))
    # scalar derivatives use every entry away from the kink
    mask = torch.from_numpy(keep).cuda()
    s_d.grad = None
    st2 = torch.tensor(step, dtype=torch.float64, requires_grad=True)
    al2 = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    out2 = prox_step(ctx, to_dev(s), to_dev(g), st2, al2)
    L2 = ((torch.conj(to_dev(c)) * out2).real * mask).sum()
    L2.backward()
    fd_step = (loss(s, g, step + h, alpha) - loss(s, g, step - h, alpha)) / (2 * h)
    fd_alpha = (loss(s, g, step, alpha + h) - loss(s, g, step, alpha - h)) / (2 * h)
    assert abs(float(st2.grad) - fd_step) <= 1e-4 * abs(fd_step) + 1e-3
    assert abs(float(al2.grad) - fd_alpha) <= 1e-4 * abs(fd_alpha) + 1e-3


def test_elastic_net_prox_step_backward_matches_fd():
    """out = shrink prox_alpha(s - step g) (the elastic-net prox, shrink = 1/(1 + eta lambda w2)):
    value against the oracle's prox of w1 ||s||_1 + (w2/2)||s||^2, and dL/dshrink, dL/dalpha and grad_s
    against FP64 central differences (entries near |z| = alpha excluded)."""
    import torch
    from oracle import Oracle
    from paper_2509_00774_gb300.autograd import prox_step
    w = W.small_T4R4_K16_16x16x8()
    ctx = make_ctx(w.geom)
    n = 3000
    s = _c64(I.complex_gaussian(n, 48))
    g = _c64(I.complex_gaussian(n, 49))
    c = _c64(I.complex_gaussian(n, 50))
    step, eta_lam, w1, w2 = 0.3, 0.5, 1.2, 0.5          # alpha = eta lambda w1, shrink = 1/(1 + eta lambda w2)
    alpha, shrink = eta_lam * w1, 1.0 / (1.0 + eta_lam * w2)
    z = s - step * g
    keep = np.abs(np.abs(z) - alpha) > 1e-2
    o = Oracle(w.geom, w1=w1, w2=w2)
    want = o.prox(z, eta_lam)
    sh = torch.tensor(shrink, dtype=torch.float64, requires_grad=True)
    al = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    s_d = to_dev(s).requires_grad_(True)
    out = prox_step(ctx, s_d, to_dev(g), step, al, sh)
    assert np.max(np.abs(to_host(out) - want)) <= 1e-5 * np.max(np.abs(want))
    mask = torch.from_numpy(keep).cuda()
    ((torch.conj(to_dev(c)) * out).real * mask).sum().backward()

    def loss(s_, al_, sh_):
        return float(np.sum((np.conj(c) * sh_ * prox_l1(s_ - step * g, al_)).real[keep]))

    h = 1e-6
    fd_sh = (loss(s, alpha, shrink + h) - loss(s, alpha, shrink - h)) / (2 * h)
    fd_al = (loss(s, alpha + h, shrink) - loss(s, alpha - h, shrink)) / (2 * h)
    assert abs(float(sh.grad) - fd_sh) <= 1e-4 * abs(fd_sh) + 1e-3
    assert abs(float(al.grad) - fd_al) <= 1e-4 * abs(fd_al) + 1e-3
    gs = to_host(s_d.grad)
    for j in np.flatnonzero(keep)[:: max(1, keep.sum() // 30)]:
        e = np.zeros(n, dtype=np.complex128)
        e[j] = h
        fd = (loss(s + e, alpha, shrink) - loss(s - e, alpha, shrink)) / (2 * h) + \
            1j * (loss(s + 1j * e, alpha, shrink) - loss(s - 1j * e, alpha, shrink)) / (2 * h)
        assert abs(gs[j] - fd) <= 1e-4 * max(1.0, abs(fd)), (j, gs[j], fd)


def _oracle_unrolled(o, y, batches, eta, lam, s_ref):
    s = np.zeros(o.N, dtype=np.complex128)
    for i, b in enumerate(batches):
        s = o.spgm_step(y, s, b, eta[i], lam[i])
    return float(np.sum(np.abs(s - s_ref) ** 2)), s


def test_unrolled_spgm_gradients_match_fd():
    """8 unrolled SPGM iterations, loss ||s_8 - s_true||^2: autograd d/deta_i, d/dlambda_i in FP32
    kernels against FP64 central differences of the oracle's unrolled iterations."""
    import torch
    from paper_2509_00774_gb300.autograd import UnrolledSPGM
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    s_true = w.scene_vector()
    y = _c64(I.add_noise(o.forward_sparse(s_true), I.complex_gaussian(o.M, 1), 30.0))
    L = o.power_iteration(I.complex_gaussian(o.N, 3), 50)
    eta0, lam0 = float(np.float32(0.8 / L)), float(np.float32(0.05 * o.lambda_max(y)))
    perm = np.concatenate([I.epoch_permutation(o.P, 2, 0), I.epoch_permutation(o.P, 2, 1)])
    batches = [perm[4 * i:4 * i + 4] for i in range(8)]
    ctx = make_ctx(w.geom)
    model = UnrolledSPGM(ctx, 8, eta0, lam0, checkpoint=True)
    with torch.no_grad():
        model.eta.copy_(torch.tensor(eta0 * (1 + 0.05 * np.arange(8)), dtype=torch.float64))
        model.lam.copy_(torch.tensor(lam0 * (1 - 0.03 * np.arange(8)), dtype=torch.float64))
    s8 = model(to_dev(y), [to_dev(b, "int32") for b in batches])
    loss = (s8 - to_dev(s_true)).abs().pow(2).sum()
    loss.backward()
    g_eta = model.eta.grad.numpy().copy()
    g_lam = model.lam.grad.numpy().copy()
    eta = model.eta.detach().numpy().astype(np.float64)
    lam = model.lam.detach().numpy().astype(np.float64)
    L0, s_orc = _oracle_unrolled(o, y, batches, eta, lam, s_true)
    assert abs(float(loss.detach()) - L0) <= 1e-4 * L0
    fd_eta, fd_lam = np.zeros(8), np.zeros(8)
    for i in range(8):
        he, hl = 1e-5 * eta[i], 1e-5 * lam[i]
        e1, e2 = eta.copy(), eta.copy()
        e1[i] += he
        e2[i] -= he
        fd_eta[i] = (_oracle_unrolled(o, y, batches, e1, lam, s_true)[0] -
                     _oracle_unrolled(o, y, batches, e2, lam, s_true)[0]) / (2 * he)
        l1, l2 = lam.copy(), lam.copy()
        l1[i] += hl
        l2[i] -= hl
        fd_lam[i] = (_oracle_unrolled(o, y, batches, eta, l1, s_true)[0] -
                     _oracle_unrolled(o, y, batches, eta, l2, s_true)[0]) / (2 * hl)
    err_eta = np.linalg.norm(g_eta - fd_eta) / np.linalg.norm(fd_eta)
    err_lam = np.linalg.norm(g_lam - fd_lam) / np.linalg.norm(fd_lam)
    print(f"[parity] unrolled grads: rel err eta {err_eta:.2e}, lambda {err_lam:.2e}")
    assert err_eta <= 1e-3 and err_lam <= 1e-3


def test_checkpointing_gives_identical_gradients():
    import torch
    from paper_2509_00774_gb300.autograd import UnrolledSPGM
    w = W.small_T4R4_K16_16x16x8()
    o = Oracle(w.geom)
    y = _c64(I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, 1), 30.0))
    ctx = make_ctx(w.geom)
    batches = [to_dev(I.epoch_permutation(o.P, 2, 0)[4 * i:4 * i + 4], "int32") for i in range(4)]
    grads = []
    for ck in (True, False):
        m = UnrolledSPGM(ctx, 8, 0.01, 0.05, checkpoint=ck)
        out = m(to_dev(y), batches)
        out.abs().pow(2).sum().backward()
        grads.append((m.eta.grad.clone(), m.lam.grad.clone()))
    assert torch.equal(grads[0][0], grads[1][0]) and torch.equal(grads[0][1], grads[1][1])


def test_unrolled_batch_of_four_scenes_mid_geometry():
    """Config-2 geometry (N = 131072), 4 scenes, 8 unrolled iterations of 16-pair minibatches."""
    import time
    import torch
    from paper_2509_00774_gb300.autograd import UnrolledSPGM
    w = W.mid_T16R16_K64_64x64x32()
    ctx = make_ctx(w.geom)
    P = w.geom.P
    all_pairs = to_dev(np.arange(P), "int32")
    ys = []
    for sc in range(4):
        s_true = to_dev(I.point_scene(w.geom.grid, 100, 200 + sc))
        ys.append(ctx.forward(all_pairs, s_true))
    y = torch.stack(ys)
    batches = [to_dev(I.epoch_permutation(P, 7, 0)[16 * i:16 * i + 16], "int32") for i in range(8)]
    model = UnrolledSPGM(ctx, 8, 0.02, 0.02, checkpoint=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = model(y, batches)
    loss = out.abs().pow(2).sum()
    loss.backward()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(f"[timing] unrolled 8 iterations x 4 scenes, forward + backward with checkpointing: {dt * 1e3:.1f} ms")
    assert out.shape == (4, w.geom.N)
    assert torch.isfinite(model.eta.grad).all() and torch.isfinite(model.lam.grad).all()


@pytest.mark.parametrize("n,offset", [(2048, 0), (1001, 0), (1001, 1), (1, 0)])
def test_prox_step_forward_matches_oracle_prox(n, offset):
    """The stand-alone step + prox kernel (16-byte path for aligned even-length vectors, element path
    for an odd tail or an 8-byte aligned view) equals the oracle's prox of s - step g."""
    import torch
    from paper_2509_00774_gb300.nfmimo import Context
    ctx = Context(0)
    rng = np.random.default_rng(n + offset)
    s = (rng.standard_normal(n + offset) + 1j * rng.standard_normal(n + offset)).astype(np.complex64)
    g = (rng.standard_normal(n + offset) + 1j * rng.standard_normal(n + offset)).astype(np.complex64)
    s_d, g_d = to_dev(s)[offset:], to_dev(g)[offset:]
    out = torch.empty(n + offset, dtype=torch.complex64, device="cuda")[offset:]
    ctx.prox_step(s_d, g_d, 0.375, 0.8, out)
    z = s[offset:].astype(np.complex128) - 0.375 * g[offset:].astype(np.complex128)
    want = prox_l1(z, 0.8)
    got = out.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - want)) <= 1e-5 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("dims", [(16, 16, 8), (15, 13, 5)])
def test_group_prox_step_matches_oracle_and_fd(dims):
    """out = shrink G_{alpha_g}(prox_alpha(s - step g)) over the 2 x 2 x 1 voxel blocks (the prox of the
    sparse-group penalty): value against the oracle's prox, and grad_s, grad_g, dL/dstep, dL/dalpha,
    dL/dalpha_g and dL/dshrink against FP64 central differences of the oracle's prox (voxels near
    |z| = alpha and blocks near ||u_b|| = alpha_g excluded).  The 15 x 13 x 5 grid has edge blocks of
    one and two voxels."""
    import torch
    from oracle import group_norms, prox_group, voxel_groups
    from paper_2509_00774_gb300.autograd import prox_step
    w = W.small_T4R4_K16_16x16x8()
    g0 = w.geom.grid
    grid = I.Grid(g0.x0, g0.y0, g0.z0, g0.dx, g0.dy, g0.dz, *dims)
    geom = I.Geometry(w.geom.tx, w.geom.rx, w.geom.freq, grid)
    ctx = make_ctx(geom)
    n = geom.N
    s = _c64(I.complex_gaussian(n, 61))
    g = _c64(I.complex_gaussian(n, 62))
    c = _c64(I.complex_gaussian(n, 63))
    step, alpha, alpha_g, shrink = 0.3, 0.4, 0.9, 0.8
    groups = voxel_groups(grid)

    def prox(s_, g_, st, al, ag, sh):
        return sh * prox_group(prox_l1(s_ - st * g_, al), groups, ag)

    z = s - step * g
    u = prox_l1(z, alpha)
    nb = group_norms(u, groups)
    keep = (np.abs(np.abs(z) - alpha) > 1e-2) & (np.abs(nb[groups] - alpha_g) > 1e-2)
    want = prox(s, g, step, alpha, alpha_g, shrink)
    zero_blocks = int(np.sum(nb <= alpha_g))
    assert 0 < zero_blocks < nb.size                       # both branches of the block shrink are taken
    pars = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in (step, alpha, alpha_g, shrink)]
    s_d = to_dev(s).requires_grad_(True)
    g_d = to_dev(g).requires_grad_(True)
    out = prox_step(ctx, s_d, g_d, pars[0], pars[1], pars[3], alpha_g=pars[2])
    assert np.max(np.abs(to_host(out) - want)) <= 1e-5 * np.max(np.abs(want))
    # keep whole blocks: a voxel's gradient depends on its block's other voxels
    keep_blocks = np.bincount(groups, weights=(~keep).astype(float), minlength=nb.size) == 0
    keep = keep_blocks[groups]
    mask = torch.from_numpy(keep).cuda()
    ((torch.conj(to_dev(c)) * out).real * mask).sum().backward()

    def loss(s_=s, g_=g, st=step, al=alpha, ag=alpha_g, sh=shrink):
        return float(np.sum((np.conj(c) * prox(s_, g_, st, al, ag, sh)).real[keep]))

    h = 1e-6
    for i, name in enumerate(("st", "al", "ag", "sh")):
        base = {"st": step, "al": alpha, "ag": alpha_g, "sh": shrink}
        up, dn = dict(base), dict(base)
        up[name] += h
        dn[name] -= h
        fd = (loss(**up) - loss(**dn)) / (2 * h)
        assert abs(float(pars[i].grad) - fd) <= 1e-4 * abs(fd) + 1e-3, (name, float(pars[i].grad), fd)
    gs, gg = to_host(s_d.grad), to_host(g_d.grad)
    for j in np.flatnonzero(keep)[:: max(1, keep.sum() // 25)]:
        e = np.zeros(n, dtype=np.complex128)
        e[j] = h
        fd_s = (loss(s_=s + e) - loss(s_=s - e)) / (2 * h) + 1j * (loss(s_=s + 1j * e) - loss(s_=s - 1j * e)) / (2 * h)
        fd_g = (loss(g_=g + e) - loss(g_=g - e)) / (2 * h) + 1j * (loss(g_=g + 1j * e) - loss(g_=g - 1j * e)) / (2 * h)
        assert abs(gs[j] - fd_s) <= 1e-4 * max(1.0, abs(fd_s)), (j, gs[j], fd_s)
        assert abs(gg[j] - fd_g) <= 1e-4 * max(1.0, abs(fd_g)), (j, gg[j], fd_g)
    print(f"[parity] group prox step {dims}: {zero_blocks} of {nb.size} blocks zero")


def test_unrolled_spgm_with_group_term_matches_oracle_iterations():
    """Unrolled SPGM with R = w1 ||s||_1 + w3 sum_b ||s_b||_2: the iterate after 6 iterations against the
    oracle's SPGM steps with the same regulariser, and finite eta / lambda gradients."""
    import torch
    from paper_2509_00774_gb300.autograd import UnrolledSPGM
    w = W.small_T4R4_K16_16x16x8()
    w1, w3 = 1.0, 0.7
    o = Oracle(w.geom, w1=w1, w3=w3)
    y = _c64(I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, 1), 30.0))
    L = o.power_iteration(I.complex_gaussian(o.N, 3), 50)
    eta, lam = 0.25 / L, float(np.float32(0.3 * o.lambda_max(y)))    # 64 of the 512 blocks vanish
    batches = [I.epoch_permutation(o.P, 7, 0)[4 * i:4 * i + 4] for i in range(4)]
    ctx = make_ctx(w.geom)
    model = UnrolledSPGM(ctx, 6, eta, lam, w1=w1, w3=w3)
    out = model(to_dev(y), [to_dev(b, "int32") for b in batches])
    s = np.zeros(o.N, dtype=np.complex128)
    for i in range(6):
        s = o.spgm_step(y, s, batches[i % 4], eta, lam)
    from oracle import nmse
    assert nmse(to_host(out), s) <= 1e-4
    from oracle import group_norms, voxel_groups
    assert np.sum(group_norms(s, voxel_groups(w.geom.grid)) == 0) > 0     # the group shrink zeroes blocks
    (out.abs() ** 2).sum().backward()
    assert torch.isfinite(model.eta.grad).all() and torch.isfinite(model.lam.grad).all()
