"""GPU parity of the prediction (degridding) path: rick_bin_predict +
rick_model_to_wplanes + rick_fft_wplanes_forward + rick_degrid_binned (through
rick_predict) against the FP64 oracle's w-stacking prediction.

Bar: max|delta| / max|V_oracle| <= 1e-5 over every visibility (small cases) or
over sampled visibilities of the MeerKAT-shaped size (the oracle's per-source
form), with the model inside the field where the taper division amplifies FP32
rounding by at most ~100 (as for imaging, the division by C(p) C(q) reaches
~5e9 at the field edges of a Kaiser-Bessel kernel without padding).  Skipped
visibilities are exactly 0, and the counts match the oracle's placement.
"""
import numpy as np
import pytest

from tests.gpu_util import oracle_config, plan_config, to_device
from visgen.workloads import meerkat, tiny_wstack

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def rk():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_19714_gb300 import rick
    rick.load()
    return rick


def _inner_model(N, C, seed, n_src=6, smooth=True):
    """Real model images [C, N, N]: point sources and (optionally) a smooth
    random component, inside the inner half of the field."""
    g = np.random.default_rng(seed)
    J = np.zeros((C, N, N), np.float32)
    for c in range(C):
        pq = g.integers(N // 4 + 1, 3 * N // 4 - 1, size=(n_src, 2))
        np.add.at(J[c], (pq[:, 1], pq[:, 0]), g.uniform(0.2, 1.0, n_src).astype(np.float32))
        if smooth:
            blob = g.standard_normal((N // 2, N // 2)).astype(np.float32) * 0.01
            J[c, N // 4:3 * N // 4, N // 4:3 * N // 4] += blob
    return J


def _gpu_predict(rk, plan, dev, J, C):
    import torch
    vis = torch.full((dev["nrow"], C), 7.0 + 7.0j, dtype=torch.complex64, device="cuda")
    counts = torch.empty(2, dtype=torch.int64, device="cuda")
    plan.predict(dev["uvw"], dev["chan_scale"], dev["weight"], dev["flag"], dev["nrow"],
                 torch.from_numpy(J).cuda(), vis, counts)
    torch.cuda.synchronize()
    plan.sync_status()
    return vis.cpu().numpy(), counts.cpu().numpy()


@pytest.mark.parametrize("fft", ["cufft", "own"])
@pytest.mark.parametrize("fold", [False, True])
def test_tiny_prediction_matches_oracle(rk, orc, fold, fft):
    img, obs = tiny_wstack(51, nvis=8000, N=256)
    obs.flag = np.zeros_like(obs.weight, dtype=np.uint8)
    obs.flag[::17] = 1
    obs.weight[5::23] = 0.0
    obs.uvw[7::41, 0] *= 1.7   # some footprints off the grid
    J = _inner_model(img.N, 1, 51)
    plan = rk.Plan(plan_config(img, 1, hermitian_fold=fold, fft_impl=fft))
    V, counts = _gpu_predict(rk, plan, to_device(obs), J, 1)
    cfg = oracle_config(orc, img)
    Vo = orc.predict(cfg, obs.uvw, obs.chan_scale, obs.weight, obs.flag, image=J[0].astype(np.float64))
    st = orc.place(cfg, obs.uvw, obs.chan_scale, obs.weight, obs.flag)["status"][:, 0]
    assert counts.tolist() == [(st == 1).sum(), (st == -1).sum()] and (st == -1).sum() > 0
    assert np.all(V[st != 1, 0] == 0)
    err = np.abs(V[:, 0] - Vo).max() / np.abs(Vo).max()
    print(f"fold={fold} fft={fft}: max|dV|/max|V| = {err:.2e}")
    assert err <= TOL


@pytest.mark.parametrize("fft", ["cufft", "own"])
@pytest.mark.parametrize("fold", [False, True])
def test_multichannel_kaiser_bessel_prediction(rk, orc, fold, fft):
    """MeerKAT-shaped, 4 channels with uneven flags, KB S = 8, odd plane count."""
    img, obs = meerkat(52, n_ant=12, n_steps=97, nchan=4, N=512, Nw=7, n_src=20)
    J = _inner_model(img.N, 4, 52)
    plan = rk.Plan(plan_config(img, 4, fft_batch=3, hermitian_fold=fold, fft_impl=fft))
    V, _ = _gpu_predict(rk, plan, to_device(obs), J, 4)
    cfg = oracle_config(orc, img)
    for c in (0, 3):
        Vo = orc.predict(cfg, obs.uvw, obs.chan_scale, obs.weight, obs.flag, channel=c,
                         image=J[c].astype(np.float64))
        err = np.abs(V[:, c] - Vo).max() / np.abs(Vo).max()
        print(f"fold={fold} channel {c}: {err:.2e}")
        assert err <= TOL


@pytest.mark.parametrize("fft", ["cufft", "own"])
def test_plane_group_streaming_gives_the_same_prediction(rk, fft):
    img, obs = meerkat(53, n_ant=10, n_steps=60, nchan=3, N=256, Nw=6, n_src=10)
    J = _inner_model(img.N, 3, 53)
    dev = to_device(obs)
    outs = []
    for budget in (0, 2 * img.N * img.N * 8, img.N * img.N * 8 * img.Nw):
        plan = rk.Plan(plan_config(img, 3, grid_budget_bytes=budget, hermitian_fold=True, fft_impl=fft))
        outs.append(_gpu_predict(rk, plan, dev, J, 3)[0])
    for o in outs[1:]:
        assert np.abs(o - outs[0]).max() <= TOL * np.abs(outs[0]).max()


@pytest.mark.parametrize("fft", ["cufft", "own"])
def test_meerkat_size_prediction_at_sampled_visibilities(rk, orc, fft):
    """The bench workload's grid (4096^2, 32 planes folded to 16, KB S = 8, FoV
    1.5 deg) on 2 channels and a point-source model of 40 sources in the inner
    field; 3000 sampled visibilities per channel against the oracle's
    per-source prediction."""
    img, obs = meerkat(54, n_steps=120, nchan=2)
    g = np.random.default_rng(54)
    N = img.N
    pq = np.unique(g.integers(N // 4, 3 * N // 4, size=(40, 2)), axis=0)
    flux = g.uniform(0.05, 1.0, len(pq)).astype(np.float32)
    J = np.zeros((2, N, N), np.float32)
    for c in range(2):
        J[c][pq[:, 1], pq[:, 0]] = flux
    plan = rk.Plan(plan_config(img, 2, hermitian_fold=True, fft_impl=fft))
    V, _ = _gpu_predict(rk, plan, to_device(obs), J, 2)
    cfg = oracle_config(orc, img)
    rows = g.choice(obs.nrow, 3000, replace=False)
    for c in range(2):
        Vo = orc.predict_at(cfg, obs.uvw, obs.chan_scale, obs.weight, obs.flag, channel=c,
                            p=pq[:, 0], q=pq[:, 1], flux=flux.astype(np.float64), rows=rows)
        err = np.abs(V[rows, c] - Vo).max() / np.abs(Vo).max()
        print(f"channel {c}: {err:.2e}")
        assert err <= TOL


@pytest.mark.parametrize("fft", ["cufft", "own"])
def test_gpu_prediction_is_the_adjoint_of_gpu_imaging(rk, fft):
    """sum_v W V conj(pred(J)) = sum W * sum_p J(p) Re I(V)(p) / n(p)^2 with both
    sides computed by the library (J real, so the real image suffices for the
    real part of the identity)."""
    import torch
    img, obs = tiny_wstack(55, nvis=20_000, N=256)
    g = np.random.default_rng(55)
    obs.vis = (g.standard_normal(obs.vis.shape) + 1j * g.standard_normal(obs.vis.shape)).astype(np.complex64)
    J = _inner_model(img.N, 1, 55)
    plan = rk.Plan(plan_config(img, 1, hermitian_fold=True, fft_impl=fft))
    dev = to_device(obs)
    P, _ = _gpu_predict(rk, plan, dev, J, 1)
    image = torch.zeros((1, img.N, img.N), dtype=torch.float32, device="cuda")
    wsum = torch.empty(1, dtype=torch.float64, device="cuda")
    plan.dirty_image(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], dev["flag"],
                     dev["nrow"], image, weight_sum=wsum)
    I = image.cpu().numpy()[0].astype(np.float64)
    N = img.N
    l = (np.arange(N) - N // 2) * img.fov / N
    n2 = 1.0 - l[None, :] ** 2 - l[:, None] ** 2
    lhs = np.real(np.sum(obs.weight[:, 0] * obs.vis[:, 0].astype(np.complex128) * np.conj(P[:, 0])))
    rhs = wsum.item() * np.sum(J[0] * I / n2)
    assert abs(lhs - rhs) <= 1e-5 * np.sum(np.abs(J[0] * I / n2)) * wsum.item()


@pytest.mark.parametrize("kw", [dict(), dict(hermitian_fold=True),
                                dict(hermitian_fold=True, w_support=4, w_kernel_param=8.0)])
def test_pruned_fused_model_transform(rk, kw):
    """rick_model_fft_wplanes pruned to the prediction binning writes only the
    reached tiles (grids filled with NaN beforehand): the degridded prediction
    equals the unpruned call's bit for bit with no NaN reaching it (with a
    w-kernel the degridder adds the Sw planes' parts with atomics, whose order
    varies from run to run: equal within 1e-6 of max|V| there), and the
    unpruned call equals rick_model_to_wplanes + rick_fft_wplanes_forward
    within FP32 rounding (2e-6 of max|V|)."""
    import torch
    img, obs = meerkat(57, n_ant=8, n_steps=30, nchan=3, N=1024, Nw=24, n_src=10)
    x = obs.uvw[:, :2] * obs.chan_scale.max() * img.fov
    obs.uvw[:, :2] *= 0.3 * img.N / np.abs(x).max()      # footprints in the central 60 %
    dev = to_device(obs)
    C, N = 3, img.N
    plan = rk.Plan(plan_config(img, C, fft_impl="own", **kw))
    ns = plan.cfg.stored_planes
    J = torch.from_numpy(_inner_model(N, C, 57)).cuda()
    plan.bin_predict(dev["uvw"], dev["chan_scale"], dev["weight"], dev["flag"], dev["nrow"])
    out = {}
    for mode in ("pruned", "full", "separate"):
        g = torch.full((C, ns, N, N), float("nan") if mode == "pruned" else 0.0,
                       dtype=torch.complex64, device="cuda")
        if mode == "separate":
            plan.model_to_wplanes(J, 0, C, 0, ns, g)
            plan.fft_wplanes_forward(g, C * ns)
        else:
            plan.model_fft_wplanes(J, 0, C, 0, ns, g, pruned=mode == "pruned")
        v = torch.zeros((dev["nrow"], C), dtype=torch.complex64, device="cuda")
        plan.degrid_binned(g, 0, C, 0, ns, v)
        torch.cuda.synchronize()
        out[mode] = v.cpu().numpy()
        if mode == "pruned":
            nan_frac = torch.isnan(g.real).float().mean().item()
            print(kw, "unwritten cells", nan_frac)
            assert nan_frac > 0.5
    assert np.isfinite(out["pruned"]).all()
    if kw.get("w_support", 0) >= 2:
        assert np.abs(out["pruned"] - out["full"]).max() <= 1e-6 * np.abs(out["full"]).max()
    else:
        np.testing.assert_array_equal(out["pruned"], out["full"])
    peak = np.abs(out["separate"]).max()
    err = np.abs(out["full"] - out["separate"]).max() / peak
    print(kw, "fused vs separate", err)
    assert err <= 2e-6


def test_prediction_rejects_the_learned_kernel_and_needs_its_binning(rk):
    import torch
    img, obs = tiny_wstack(56, nvis=100, N=128)
    dev = to_device(obs)
    plan = rk.Plan(plan_config(img, 1))
    grids = torch.empty((1, img.Nw, img.N, img.N), dtype=torch.complex64, device="cuda")
    vis = torch.zeros((dev["nrow"], 1), dtype=torch.complex64, device="cuda")
    wsum = torch.empty(1, dtype=torch.float64, device="cuda")
    plan.bin(dev["uvw"], dev["chan_scale"], dev["vis"], dev["weight"], None, dev["nrow"], wsum)
    with pytest.raises(rk.RickError):
        plan.degrid_binned(grids, 0, 1, 0, img.Nw, vis)   # binned for gridding, not prediction
    plan.bin_predict(dev["uvw"], dev["chan_scale"], dev["weight"], None, dev["nrow"])
    with pytest.raises(rk.RickError):
        plan.grid_binned(0, 1, 0, img.Nw, grids)           # binned for prediction
    limg = img.with_(S=4, kernel="learned", kernel_param=5.6)
    lplan = rk.Plan(plan_config(limg, 1))
    with pytest.raises(rk.RickError) as e:
        lplan.bin_predict(dev["uvw"], dev["chan_scale"], dev["weight"], None, dev["nrow"])
    assert e.value.status == 6
