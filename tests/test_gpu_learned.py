"""Learned support-4 kernel (pattern 4) on the GPU: the network's forward and
backward kernels against the FP64 oracle network, the baked correction table,
gridding with Kaiser-Bessel taps plus the table against the oracle's learned
kernel (and, for a zero table, against plain Kaiser-Bessel gridding), the
training objective (image and direct inversion at the probes) against the
oracle, the training gradient against finite differences of the oracle's
loss, what training gains over the untrained start (exactly the support-4
Kaiser-Bessel) on held-out fields, and checkpoint/resume."""
import numpy as np
import pytest

import visgen
from tests.gpu_util import assert_image_close, plan_config, run_path, to_device
from visgen.workloads import KB_BETA_S4, learned_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rk():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2601_19714_gb300 import rick
    rick.load()
    return rick


def _learn_cfg(rk, img):
    return rk.Config(N=img.N, n_wplanes=img.Nw, support=4, n_channels=1, fov_rad=img.fov,
                     w_min=img.w_min, w_max=img.w_max, kernel="table", kernel_param=KB_BETA_S4)


@pytest.mark.parametrize("H", [16, 64])
def test_mlp_forward_and_backward_match_oracle(rk, orc, H):
    import torch
    from paper_2601_19714_gb300 import learned
    prm = learned.init_params(H, 3)
    n = 37
    x = np.random.default_rng(1).random((n, 3)).astype(np.float32)
    gout = np.random.default_rng(2).normal(size=(n, 16)).astype(np.float32)
    dp, dx = torch.from_numpy(prm).cuda(), torch.from_numpy(x).cuda()
    out = torch.empty((n, 16), device="cuda")
    rk.mlp_forward(dp, H, dx, out)
    ref = np.stack([orc.mlp_forward(prm.astype(np.float64), H, xi.astype(np.float64)) for xi in x])
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()
    grad = torch.zeros(prm.size, device="cuda")
    rk.mlp_backward(dp, H, dx, torch.from_numpy(gout).cuda(), grad,
                    torch.empty((n, 6 * H), device="cuda"), torch.empty((n, 16), device="cuda"))
    gref = sum(orc.mlp_backward(prm.astype(np.float64), H, xi.astype(np.float64),
                                gi.astype(np.float64)) for xi, gi in zip(x, gout))
    assert np.abs(grad.cpu().numpy() - gref).max() <= 1e-5 * np.abs(gref).max()


def test_baked_table_is_the_network_on_the_lattice(rk, orc):
    from paper_2601_19714_gb300 import learned
    k = learned.LearnedKernel(5, 32, 8, seed=4)
    tab = k.bake().cpu().numpy().reshape(5, 9, 9, 16)
    prm = k.params.cpu().numpy().astype(np.float64)
    for kk in (0, 2, 4):
        for iy in (0, 3, 8):
            for ix in (0, 5, 8):
                ref = orc.mlp_forward(prm, 32, [ix / 8, iy / 8, (2 * kk - 4) / 4])
                np.testing.assert_allclose(tab[kk, iy, ix], ref, atol=1e-5 * np.abs(ref).max())


def test_gridding_with_the_table_matches_the_oracle_learned_kernel(rk, orc):
    """Kaiser-Bessel taps plus the table through rick_grid / FFT / phase
    against the oracle's learned kernel (the same network evaluated in FP64
    on the same lattice)."""
    import torch
    from paper_2601_19714_gb300 import learned
    img, obs = learned_field(21, nvis=30_000, N=256, Nw=8, n_src=6)
    k = learned.LearnedKernel(img.Nw, 64, 16, seed=9, zero_output=False)
    with torch.no_grad():
        k.params[-(16 * 64 + 16):] *= 0.01   # a small correction, as after training
    plan = rk.Plan(plan_config(img, 1))
    plan.set_kernel_table(k.bake(), 16)
    I_g, _, _, _ = run_path(plan, to_device(obs), 1, img.N, img.Nw)
    ocfg = orc.Config(img.N, img.Nw, 4, "learned", KB_BETA_S4, img.fov, img.w_min, img.w_max,
                      mlp=k.params.cpu().numpy().astype(np.float64), mlp_hidden=64, mlp_lattice=16)
    I_o, _ = orc.image(ocfg, obs.uvw, obs.chan_scale, obs.vis, obs.weight)
    assert_image_close(I_g[0], I_o.real, plan.taper(), 1e-5)


def test_table_set_after_binning_applies_to_the_next_gridding(rk):
    """The correction taps are interpolated per record at each gridding call,
    so a table set between rick_bin and rick_grid_binned is the one used: the
    planes equal those of a plan that had that table from the start (to FP32
    rounding)."""
    import torch
    from paper_2601_19714_gb300 import learned
    img, obs = learned_field(23, nvis=30_000, N=256, Nw=8, n_src=5)
    dev = to_device(obs)
    tabs = []
    for seed in (3, 4):
        k = learned.LearnedKernel(img.Nw, 64, 16, seed=seed, zero_output=False)
        with torch.no_grad():
            k.params[-(16 * 64 + 16):] *= 0.01
        tabs.append(k.bake().clone())
    N, Nw = img.N, img.Nw
    ws = torch.empty(1, dtype=torch.float64, device="cuda")
    planes = []
    for first, second in ((0, 1), (1, None)):
        plan = rk.Plan(plan_config(img, 1))
        plan.set_kernel_table(tabs[first], 16)
        g = torch.empty((1, Nw, N, N), dtype=torch.complex64, device="cuda")
        plan.grid(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], None, obs.nrow, 0, Nw, g, ws)
        if second is not None:
            plan.set_kernel_table(tabs[second], 16)
            plan.grid_binned(0, 1, 0, Nw, g)
        torch.cuda.synchronize()
        planes.append(g.cpu().numpy())
    # two binnings: the record order within a bin follows the atomics, so the
    # FP32 sums agree to rounding, not bit for bit
    peak = np.abs(planes[1]).max()
    assert peak > 0
    assert np.abs(planes[0] - planes[1]).max() <= 1e-6 * peak


def test_zero_correction_is_exactly_kaiser_bessel(rk):
    """The untrained learned kernel (zero output layer) grids exactly like the
    support-4 Kaiser-Bessel kernel."""
    from paper_2601_19714_gb300 import learned
    img, obs = learned_field(22, nvis=20_000, N=256, Nw=8, n_src=4)
    k = learned.LearnedKernel(img.Nw, 64, 16, seed=1)
    assert float(k.bake().abs().max()) == 0.0
    p_tab = rk.Plan(plan_config(img, 1))
    p_tab.set_kernel_table(k.table, 16)
    p_kb = rk.Plan(plan_config(img.with_(kernel="kb"), 1))
    I_t, _, _, _ = run_path(p_tab, to_device(obs), 1, img.N, img.Nw)
    I_k, _, _, _ = run_path(p_kb, to_device(obs), 1, img.N, img.Nw)
    assert_image_close(I_t[0], I_k[0], p_kb.taper(), 1e-6)


def _field_setup(rk, seed=5, nvis=20_000, N=256, Nw=8, L=16):
    img, obs = learned_field(seed, nvis=nvis, N=N, Nw=Nw, n_src=3)
    dev = to_device(obs)
    learn = rk.Learn(_learn_cfg(rk, img), L, dev["uvw"], dev["weight"][:, 0].contiguous())
    return img, obs, learn


def _oracle_loss(orc, img, obs, params64, L, src):
    N = img.N
    dl = img.fov / N
    lm = np.concatenate([(src[:, :2] - N // 2) * dl, src[:, 2:3]], axis=1)
    vis = visgen.predict(obs.uvw, obs.chan_scale, lm)
    cfg = orc.Config(N, img.Nw, 4, "learned", KB_BETA_S4, img.fov, img.w_min, img.w_max,
                     mlp=params64, mlp_hidden=_hidden(params64), mlp_lattice=L)
    p, q = src[:, 0].astype(np.int32), src[:, 1].astype(np.int32)
    I = orc.image_at(cfg, obs.uvw, obs.chan_scale, vis, obs.weight, None, 0, p, q).real
    D = orc.dft_at(cfg, obs.uvw, obs.chan_scale, vis, obs.weight, None, 0, p, q).real
    return ((I - D) ** 2).sum() / (D ** 2).sum(), I, D


def _hidden(params):
    # 3H + H + H^2 + H + 16H + 16 = n  ->  H^2 + 21 H + 16 - n = 0
    n = params.size
    return int(round((-21 + np.sqrt(21 * 21 - 4 * (16 - n))) / 2))


def test_training_objective_matches_oracle(rk, orc):
    import torch
    from paper_2601_19714_gb300 import learned
    img, obs, learn = _field_setup(rk)
    assert learn.placed() == obs.nrow
    k = learned.LearnedKernel(img.Nw, 64, 16, seed=7, zero_output=False)
    k.bake()
    src = learned.training_field(11, img.N)[:6]
    idft = torch.zeros((64, 2), device="cuda")
    learn.field_grad(k.table, src, src[:, :2].astype(np.int32), None, k.loss, idft)
    got = idft.cpu().numpy()[:len(src)]
    loss_o, I_o, D_o = _oracle_loss(orc, img, obs, k.params.cpu().numpy().astype(np.float64), 16, src)
    scale = np.abs(D_o).max()
    assert np.abs(got[:, 0] - I_o).max() <= 1e-5 * max(scale, np.abs(I_o).max())
    assert np.abs(got[:, 1] - D_o).max() <= 1e-5 * scale
    assert k.loss.item() == pytest.approx(loss_o, rel=1e-4)


def test_training_gradient_matches_finite_differences_of_the_oracle(rk, orc):
    """d loss / d params from the GPU kernels (objective backward, then the
    network backward) against central differences of the oracle's FP64 loss."""
    from paper_2601_19714_gb300 import learned
    img, obs, learn = _field_setup(rk, seed=8, nvis=3000, N=128, Nw=4, L=8)
    k = learned.LearnedKernel(img.Nw, 16, 8, seed=3, zero_output=False)
    src = learned.training_field(13, img.N)[:4]
    k.bake()
    learn.field_grad(k.table, src, src[:, :2].astype(np.int32), k.table_grad, k.loss)
    k.grad.zero_()
    rk.mlp_backward(k.params, 16, k.lattice_in, k.table_grad, k.grad, k.work, k.scratch)
    g = k.grad.cpu().numpy().astype(np.float64)
    p0 = k.params.cpu().numpy().astype(np.float64)
    for i in np.argsort(-np.abs(g))[:6]:
        h = 1e-4 * max(1.0, abs(p0[i]))
        pp, pm = p0.copy(), p0.copy()
        pp[i] += h
        pm[i] -= h
        fd = (_oracle_loss(orc, img, obs, pp, 8, src)[0] - _oracle_loss(orc, img, obs, pm, 8, src)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=2e-2, abs=1e-3 * np.abs(g).max()), (i, g[i], fd)


def test_training_beats_the_untrained_kernel(rk):
    """What the network gains: 64 held-out fields (sources at continuous
    positions, judged at 64 pixels of the taper-gated field) imaged with the
    trained kernel against the untrained one, which is exactly the support-4
    Kaiser-Bessel (the method without the learned part).  The network is
    trained on 9,600 other fields (600 Adam steps of 16)."""
    from paper_2601_19714_gb300 import learned
    img, obs, learn = _field_setup(rk, seed=5, nvis=60_000, N=256, Nw=8, L=16)
    k = learned.LearnedKernel(img.Nw, 64, 16, seed=7)
    base = k.losses(learn, 64)
    k.train(learn, 600, lr=3e-5, batch=16)
    after = k.losses(learn, 64)
    gain_mean = 1.0 - after.mean() / base.mean()
    gain_median = 1.0 - np.median(after) / np.median(base)
    better = float((after < base).mean())
    print(f"held-out loss mean {base.mean():.3e} -> {after.mean():.3e} ({100 * gain_mean:.1f} %), "
          f"median {np.median(base):.3e} -> {np.median(after):.3e} ({100 * gain_median:.1f} %), "
          f"fields better {100 * better:.0f} %")
    assert gain_mean >= 0.05 and gain_median >= 0.03 and better >= 0.55


def test_checkpoint_resume_continues_the_same_run(rk, tmp_path):
    from paper_2601_19714_gb300 import learned
    img, obs, learn = _field_setup(rk, seed=6, nvis=8000, N=128, Nw=4, L=8)
    a = learned.LearnedKernel(img.Nw, 16, 8, seed=2)
    a.train(learn, 10, batch=4)
    path = str(tmp_path / "ckpt")
    a.save(path)
    a.train(learn, 10, batch=4)
    b = learned.LearnedKernel.load(path)
    assert (b.state.step, b.adam_t) == (40, 10)
    b.train(learn, 10, batch=4)
    assert b.state.step == a.state.step == 80
    pa, pb = a.params.cpu().numpy(), b.params.cpu().numpy()
    assert np.abs(pa - pb).max() <= 1e-3 * np.abs(pa).max()
