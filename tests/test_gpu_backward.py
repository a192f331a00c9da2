"""GPU adjoint raymarch: gradients against the FP64 oracle's gradient and against
central finite differences of the GPU forward renderer, plus the autograd
binding and a short transfer-function fit.

Bars: normwise relative error <= 1e-3 per parameter group against the
oracle (at full size, a uniform's error relative to the sum of its blocks' absolute
gradients, the scale of a float32 sum's rounding bound); rays whose stopping sample is ambiguous, or that pass within float32
rounding of a point where the sample's opacity or colour has a kink (a
transfer-function knot, a clamp; oracle FLAG_KINK), carry no upstream gradient
-- there the two one-sided derivatives are both correct -- and they are at most
5% of the rays. Directional finite differences of the FP32 forward within 1e-3
relative.
"""

import numpy as np
import pytest

import oracle
import phantoms as ph
from phantoms import workloads
from tests.gpu_util import oracle_params, torch_cuda

pytestmark = pytest.mark.gpu
TOL_GRAD = 1e-3


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def vr(torch):
    import paper_2605_19737_gb300 as pkg
    ctx = pkg.Context(0)
    yield ctx
    ctx.close()


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _setup(vr, torch, case, In):
    """Load the case's volume, then replace its intensities by In (normalised)."""
    vol = case["volume"]
    vid = vr.load_volume(torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda(),
                         case["spacing"])
    vr.set_normalized(vid, torch.from_numpy(In.astype(np.float32)).cuda())
    vr.precompute_morphology(vid, case.get("sigmas", ()))
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    return vid


def _cases():
    head = workloads.head64_128px()
    small = dict(head, volume=ph.head_phantom((28, 26, 24), seed=71), W=40, H=36,
                 cams=ph.camera_array([ph.orbit_camera((28, 26, 24), (1, 1, 1), az, el, width=40, height=36)
                                       for az, el in ((30, 20), (150, -25))]))
    small["params"] = dict(small["params"], gamma=0.4, kappa_ref=0.1, w_max=3.0)
    bw = workloads.scaled_brainweb((41, 47, 39), width=44, height=36, n_cams=2)
    corr = dict(small, params=dict(small["params"], opacity_ref_step=0.7, step_vox=0.4))
    # no curvature term: the forward never reads the Hessian, dL/dgamma still needs kappa
    flat = dict(small, params=dict(small["params"], gamma=0.0))
    return {"head_1d": small, "brainweb_2d": bw, "head_1d_corrected": corr, "head_1d_gamma0": flat}


@pytest.mark.parametrize("kernel", [0, 2, 3, "state"])  # per-lane (derived bricks), brick-synchronous,
#                                                          per-lane stencils, per-lane from the forward's ray state
@pytest.mark.parametrize("name", ["head_1d", "brainweb_2d", "head_1d_corrected", "head_1d_gamma0"])
def test_backward_matches_oracle_gradient(vr, torch, name, kernel):
    case = _cases()[name]
    In32 = oracle.normalize(case["volume"]).astype(np.float32)
    In = In32.astype(np.float64)
    vid = _setup(vr, torch, case, In32)
    _, _, gmax = vr.get_norm(vid)
    n, H, W = case["cams"].shape[0], case["H"], case["W"]
    rng = np.random.default_rng(72)
    dl = rng.normal(size=(n, H, W, 4))
    P = oracle_params(case["params"], case["tf"])
    fwd = oracle.render(In, case["spacing"], P, case["tf"], case["cams"], W, H, gmax_value=gmax, alternatives=False)
    amb = (fwd.flags & (oracle.FLAG_ET | oracle.FLAG_COUNT | oracle.FLAG_KINK)) != 0
    assert amb.mean() <= 0.05
    dl[amb] = 0.0
    dtf_o, dpar_o, dvol_o = oracle.render_grad(In, case["spacing"], P, case["tf"], case["cams"], W, H, dl,
                                               gmax_value=gmax)
    state = None
    if kernel == "state":
        state = torch.empty((n, H, W, 2), dtype=torch.float32, device="cuda")
        vr.render(vid, case["cams"], W, H, ray_state=state)
        kernel = 0
    dtf, dpar, dvol = vr.render_backward(vid, case["cams"], W, H, torch.from_numpy(dl.astype(np.float32)).cuda(),
                                         kernel=kernel, ray_state=state)
    dtf, dpar, dvol = dtf.cpu().numpy(), dpar.cpu().numpy(), dvol.cpu().numpy()
    e_tf, e_vol = _rel(dtf, dtf_o), _rel(dvol, dvol_o)
    used = [0, 1, 2, 3, 4] if case["params"]["shading"] else [0, 4]
    e_par = max(abs(dpar[k] - dpar_o[k]) / max(abs(dpar_o[k]), 1e-6 * np.abs(dpar_o).max()) for k in used)
    print("%s: rel err tf %.2e params %.2e volume %.2e (ambiguous rays %d)" % (name, e_tf, e_par, e_vol, amb.sum()))
    assert np.linalg.norm(dtf_o) > 0 and np.linalg.norm(dvol_o) > 0
    assert e_tf <= TOL_GRAD and e_par <= TOL_GRAD and e_vol <= TOL_GRAD
    vr.free_volume(vid)


@pytest.mark.parametrize("packet_w", [4, 8, 16])
def test_merged_scatter_at_dense_rays(vr, torch, packet_w):
    """Rays ~0.25 voxel apart, so that neighbouring lanes of a packet sample the same
    cell at the same step and the backward merges their channel-gradient scatter
    (horizontal pairs, then vertical pairs lane ^ packet_w), with a curvature term
    (Hessian channel gradients) and every packet shape: the gradients still match the
    oracle's."""
    base = _cases()["head_1d"]
    dims = (28, 26, 24)
    case = dict(base, W=96, H=88, cams=ph.camera_array([ph.orbit_camera(dims, (1, 1, 1), 35, 15, width=96,
                                                                         height=88, fov_deg=14.0)]))
    In32 = oracle.normalize(case["volume"]).astype(np.float32)
    In = In32.astype(np.float64)
    vid = _setup(vr, torch, case, In32)
    _, _, gmax = vr.get_norm(vid)
    n, H, W = 1, case["H"], case["W"]
    dl = np.random.default_rng(79).normal(size=(n, H, W, 4))
    P = oracle_params(case["params"], case["tf"])
    fwd = oracle.render(In, case["spacing"], P, case["tf"], case["cams"], W, H, gmax_value=gmax, alternatives=False)
    amb = (fwd.flags & (oracle.FLAG_ET | oracle.FLAG_COUNT | oracle.FLAG_KINK)) != 0
    assert amb.mean() <= 0.05
    dl[amb] = 0.0
    dtf_o, dpar_o, dvol_o = oracle.render_grad(In, case["spacing"], P, case["tf"], case["cams"], W, H, dl,
                                               gmax_value=gmax)
    state = torch.empty((n, H, W, 2), dtype=torch.float32, device="cuda")
    vr.render(vid, case["cams"], W, H, ray_state=state)
    dtf, dpar, dvol = vr.render_backward(vid, case["cams"], W, H, torch.from_numpy(dl.astype(np.float32)).cuda(),
                                         ray_state=state, packet_w=packet_w)
    dtf, dvol = dtf.cpu().numpy(), dvol.cpu().numpy()
    e_tf, e_vol = _rel(dtf, dtf_o), _rel(dvol, dvol_o)
    print("packet %d: rel err tf %.2e volume %.2e" % (packet_w, e_tf, e_vol))
    assert np.linalg.norm(dvol_o) > 0
    assert e_tf <= TOL_GRAD and e_vol <= TOL_GRAD
    vr.free_volume(vid)


@pytest.mark.parametrize("variant", ["et", "no_et", "opaque_no_et"])
def test_ray_state_replaces_the_re_march(vr, torch, variant):
    """The per-ray state the forward records (last sample, transmittance in front of
    it) gives the backward the re-march's starting point: equal gradients; with early
    termination the recorded index is the dense sample count - 1; with it off and
    fully opaque samples (A reaches 1) the sweep starts at the first of them."""
    case = _cases()["head_1d"]
    if variant != "et":
        case["params"] = dict(case["params"], et_threshold=2.0)
    if variant == "opaque_no_et":
        case["params"] = dict(case["params"], opacity_scale=60.0)
    In32 = oracle.normalize(case["volume"]).astype(np.float32)
    vid = _setup(vr, torch, case, In32)
    n, H, W = case["cams"].shape[0], case["H"], case["W"]
    state = torch.empty((n, H, W, 2), dtype=torch.float32, device="cuda")
    rs = torch.zeros((n, H, W, 2), dtype=torch.int32, device="cuda")
    img = vr.render(vid, case["cams"], W, H, ray_state=state, ray_samples=rs)
    torch.cuda.synchronize()
    kl = state[..., 0].contiguous().view(torch.int32).cpu().numpy()
    dense = rs[..., 0].cpu().numpy()
    if variant != "opaque_no_et":
        np.testing.assert_array_equal(kl, dense - 1)
    else:
        assert (kl < dense - 1).sum() > 0 and np.all(kl <= dense - 1)
        assert float(img[..., 3].max()) == 1.0
    t = state[..., 1].cpu().numpy()
    assert np.all((t >= 0.0) & (t <= 1.0))
    dl = torch.from_numpy(np.random.default_rng(75).normal(size=(n, H, W, 4)).astype(np.float32)).cuda()
    a = [x.cpu().numpy() for x in vr.render_backward(vid, case["cams"], W, H, dl)]
    b = [x.cpu().numpy() for x in vr.render_backward(vid, case["cams"], W, H, dl, ray_state=state)]
    for x, y in zip(a, b):
        # the two starting points differ only by the rounding of A (float32 contraction)
        assert np.all(np.isfinite(y))
        assert _rel(y, x) <= 1e-4
    vr.free_volume(vid)


def test_backward_matches_gpu_finite_differences(vr, torch):
    """Directional derivatives of L = sum(dl * render) by central differences of the GPU
    forward renderer (float32; early termination off so no stopping index flips)."""
    case = _cases()["head_1d"]
    # early termination off (no stopping index flips) and kappa_ref such that w(kappa)
    # rarely sits on its clamps, whose kinks a finite step would straddle
    case["params"] = dict(case["params"], et_threshold=2.0, kappa_ref=1.0)
    # no opacity entry on the clamp kink at 0, where a central difference is one-sided
    case["tf"] = case["tf"].copy()
    case["tf"][..., 3] += np.float32(0.01)
    In32 = oracle.normalize(case["volume"]).astype(np.float32)
    vid = _setup(vr, torch, case, In32)
    n, H, W = case["cams"].shape[0], case["H"], case["W"]
    rng = np.random.default_rng(73)
    dl = torch.from_numpy(rng.normal(size=(n, H, W, 4)).astype(np.float32)).cuda()

    def loss(tf=None, params=None, norm=None):
        if norm is not None:
            vr.set_normalized(vid, norm)
        vr.set_tissue_params(vid, case["tf"] if tf is None else tf, **(params or case["params"]))
        img = vr.render(vid, case["cams"], W, H)
        return float((img.double() * dl.double()).sum())

    vr.set_normalized(vid, torch.from_numpy(In32).cuda())
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    dtf, dpar, dvol = [x.cpu().numpy().astype(np.float64) for x in vr.render_backward(vid, case["cams"], W, H, dl)]
    # transfer function
    u = rng.normal(size=case["tf"].shape)
    tp = (case["tf"] + 1e-3 * u).astype(np.float32)
    tm = (case["tf"] - 1e-3 * u).astype(np.float32)
    fd = loss(tf=tp) - loss(tf=tm)
    want = float(np.sum(dtf * (tp.astype(np.float64) - tm.astype(np.float64))))
    assert fd == pytest.approx(want, rel=TOL_GRAD)
    # uniforms
    for idx, name in enumerate(["gamma", "ka", "kd", "ks", "opacity_scale"]):
        h = 1e-3
        pp = dict(case["params"], **{name: case["params"][name] + h})
        pm = dict(case["params"], **{name: case["params"][name] - h})
        rp = float(np.float32(pp[name])) - float(np.float32(pm[name]))
        fd = (loss(params=pp) - loss(params=pm)) / rp
        assert fd == pytest.approx(dpar[idx], rel=5 * TOL_GRAD, abs=1e-3 * np.abs(dpar).max()), name
    # voxels (normalised intensities), on a configuration smooth in the voxels:
    # linear transfer function, no curvature term, no shading, no gradient-magnitude
    # modulation. |grad I| is a cone at grad I = 0, and a white-noise voxel step
    # moves the gradient of the many low-|grad I| samples by a comparable amount, so
    # with those terms on, the central difference is off by ~1e-3 at any step that
    # float32 resolves (the oracle comparison above covers those terms)
    case["tf"] = np.zeros_like(case["tf"])
    x = np.arange(case["tf"].shape[1], dtype=np.float32) / (case["tf"].shape[1] - 1)
    case["tf"][0, :, 0], case["tf"][0, :, 1], case["tf"][0, :, 2] = 0.2 + 0.6 * x, 0.9 - 0.5 * x, 0.5
    case["tf"][0, :, 3] = 0.01 + 0.12 * x
    case["params"] = dict(case["params"], gamma=0.0, shading=0, grad_mod=0)
    vr.set_normalized(vid, torch.from_numpy(In32).cuda())
    vr.set_tissue_params(vid, case["tf"], **case["params"])
    _, _, dvol = [x.cpu().numpy().astype(np.float64) for x in vr.render_backward(vid, case["cams"], W, H, dl)]
    u = rng.normal(size=In32.shape)
    h = 3e-3
    vp = torch.from_numpy((In32 + h * u).astype(np.float32)).cuda()
    vm = torch.from_numpy((In32 - h * u).astype(np.float32)).cuda()
    step = (vp.double() - vm.double()).cpu().numpy()
    fd = loss(norm=vp) - loss(norm=vm)
    assert fd == pytest.approx(float(np.sum(dvol * step)), rel=TOL_GRAD)
    vr.free_volume(vid)


def test_zero_opacity_region_has_zero_voxel_gradient(vr, torch):
    case = _cases()["head_1d"]
    case["tf"] = ph.tf_constant((1, 1, 1), 0.0)
    In32 = oracle.normalize(case["volume"]).astype(np.float32)
    vid = _setup(vr, torch, case, In32)
    n, H, W = case["cams"].shape[0], case["H"], case["W"]
    dl = torch.ones((n, H, W, 4), device="cuda")
    dtf, dpar, dvol = vr.render_backward(vid, case["cams"], W, H, dl)
    assert float(dvol.abs().max()) == 0.0
    assert float(dtf[..., :3].abs().max()) == 0.0 and float(dtf[..., 3].abs().max()) > 0.0
    vr.free_volume(vid)


def test_autograd_and_short_fit(vr, torch):
    """torch.autograd through the C ABI; Adam on sigmoid-parameterised TF entries
    lowers the MSE to a target rendered from a perturbed TF."""
    from paper_2605_19737_gb300 import autograd as ag
    case = _cases()["head_1d"]
    In32 = oracle.normalize(case["volume"]).astype(np.float32)
    vid = _setup(vr, torch, case, In32)
    n, H, W = case["cams"].shape[0], case["H"], case["W"]
    fixed = {k: v for k, v in case["params"].items() if k not in ag.PARAM_NAMES}
    params = torch.tensor([case["params"][k] for k in ag.PARAM_NAMES], dtype=torch.float32)
    rng = np.random.default_rng(74)
    tf_target = np.clip(case["tf"] + rng.normal(0, 0.05, case["tf"].shape), 0, 1).astype(np.float32)
    with torch.no_grad():
        target = ag.render(vr, vid, torch.from_numpy(tf_target).cuda(), params, case["cams"], W, H, fixed)
    # gradient of the autograd path == direct call
    tf = torch.from_numpy(case["tf"]).cuda().requires_grad_(True)
    img = ag.render(vr, vid, tf, params, case["cams"], W, H, fixed)
    loss = ((img - target) ** 2).mean()
    loss.backward()
    g_direct, _, _ = vr.render_backward(vid, case["cams"], W, H, (2.0 / img.numel()) * (img - target).detach(),
                                        want_volume=False)
    np.testing.assert_allclose(tf.grad.cpu().numpy(), g_direct.cpu().numpy(), rtol=1e-5, atol=1e-9)
    # fit
    logit = torch.logit(torch.from_numpy(case["tf"]).cuda().clamp(1e-4, 1 - 1e-4)).requires_grad_(True)
    opt = torch.optim.Adam([logit], lr=1e-2)
    losses = []
    for _ in range(60):
        opt.zero_grad()
        img = ag.render(vr, vid, torch.sigmoid(logit), params, case["cams"], W, H, fixed)
        lo = ((img - target) ** 2).mean()
        lo.backward()
        opt.step()
        losses.append(float(lo.detach()))
    assert losses[-1] < 0.5 * losses[0], losses
    vr.free_volume(vid)


def test_data_parallel_fit_through_the_library(vr, torch):
    """dp_fit with the library's per-shard step (one process: every view in one
    shard) follows the plain autograd fit of the same MSE: same loss curve within
    float32 summation-order differences, and the MSE falls."""
    from paper_2605_19737_gb300 import autograd as ag
    from paper_2605_19737_gb300 import fit as fitmod
    from paper_2605_19737_gb300.distributed import dp_fit, library_shard_loss_grad
    case = _cases()["head_1d"]
    In32 = oracle.normalize(case["volume"]).astype(np.float32)
    vid = _setup(vr, torch, case, In32)
    n, H, W = case["cams"].shape[0], case["H"], case["W"]
    fixed = {k: v for k, v in case["params"].items() if k not in ag.PARAM_NAMES}
    params = torch.tensor([case["params"][k] for k in ag.PARAM_NAMES], dtype=torch.float32)
    rng = np.random.default_rng(76)
    tf_target = np.clip(case["tf"] + rng.normal(0, 0.05, case["tf"].shape), 0, 1).astype(np.float32)
    with torch.no_grad():
        target = ag.render(vr, vid, torch.from_numpy(tf_target).cuda(), params, case["cams"], W, H, fixed)
    tf0 = torch.from_numpy(case["tf"]).cuda()
    f = library_shard_loss_grad(vr, vid, case["cams"], W, H, fixed, params, target)
    x_dp, l_dp = dp_fit(f, tf0, n, steps=30, lr=1e-2)
    x_ref, l_ref, _ = fitmod.fit_transfer_function(vr, vid, case["cams"], W, H, tf0, target, fixed, params, steps=30)
    np.testing.assert_allclose(l_dp, l_ref, rtol=2e-3)
    assert np.abs(x_dp.cpu().numpy() - x_ref.cpu().numpy()).max() < 2e-3
    assert l_dp[-1] < 0.6 * l_dp[0], l_dp
    vr.free_volume(vid)


@pytest.mark.slow
@pytest.mark.parametrize("name", ["diff_head128_8cam", "brainweb_1080p"])
def test_backward_full_size_sampled(vr, torch, name):
    """Full-size workloads in the benchmark's launch configuration (the forward records
    the ray state, the backward sweeps from it): the upstream gradient lives on every
    16th pixel row and column only, and the gradients match the oracle's gradient of
    that same sampled loss (whose other rays add exactly zero)."""
    case = workloads.diff_head128_8cam() if name.startswith("diff") else workloads.brainweb_1080p()
    In32 = oracle.normalize(case["volume"]).astype(np.float32)
    vid = _setup(vr, torch, case, In32)
    _, _, gmax = vr.get_norm(vid)
    n, H, W = case["cams"].shape[0], case["H"], case["W"]
    P = oracle_params(case["params"], case["tf"])
    In = In32.astype(np.float64)
    fwd = oracle.render(In, case["spacing"], P, case["tf"], case["cams"], W, H, gmax_value=gmax, pix_stride=16,
                        alternatives=False)
    sampled = np.zeros((n, H, W), bool)
    sampled[:, ::16, ::16] = True
    amb = (fwd.flags & (oracle.FLAG_ET | oracle.FLAG_COUNT | oracle.FLAG_KINK)) != 0
    # full-length rays (hundreds of samples) meet a knot or clamp within float32
    # rounding more often than the small cases' rays: ~1 % here
    assert (amb & sampled).sum() <= 0.05 * sampled.sum()
    dl = np.random.default_rng(75).normal(size=(n, H, W, 4)).astype(np.float32)
    dl[~sampled | amb] = 0.0
    dtf_o, dpar_o, dvol_o = oracle.render_grad(In, case["spacing"], P, case["tf"], case["cams"], W, H,
                                               dl.astype(np.float64), gmax_value=gmax)
    state = torch.empty((n, H, W, 2), dtype=torch.float32, device="cuda")
    vr.render(vid, case["cams"], W, H, ray_state=state)
    dtf, dpar, dvol = vr.render_backward(vid, case["cams"], W, H, torch.from_numpy(dl).cuda(), ray_state=state)
    dtf, dpar, dvol = dtf.cpu().numpy(), dpar.cpu().numpy(), dvol.cpu().numpy()
    used = [0, 1, 2, 3, 4] if case["params"]["shading"] else [0, 4]  # d/dgamma also at gamma = 0
    # Each uniform's gradient is a sum over thousands of rays whose signs follow the random
    # upstream gradient; a float32 sum's rounding error is bounded relative to the sum of
    # the terms' magnitudes (|fl(sum x) - sum x| <= gamma_n sum |x|), not to the possibly
    # cancelling total (opacity_scale here: total 0.028 from row sums up to 2.6). The bar
    # is taken against sum |partial gradient| over 16 blocks of rays -- a lower bound of
    # sum |x|, so never looser than that bound -- from the oracle.
    rows = [(c, y) for c in range(n) for y in range(0, H, 16)]
    scale = np.zeros(5)
    for blk in np.array_split(np.arange(len(rows)), 16):
        d1 = np.zeros_like(dl)
        for r in blk:
            d1[rows[r]] = dl[rows[r]]
        _, pb, _ = oracle.render_grad(In, case["spacing"], P, case["tf"], case["cams"], W, H,
                                      d1.astype(np.float64), gmax_value=gmax, want_volume=False)
        scale += np.abs(pb)
    assert np.all(scale >= np.abs(dpar_o) * (1 - 1e-12))
    e_par = max(abs(dpar[k] - dpar_o[k]) / max(scale[k], 1e-30) for k in used)
    e_tf, e_vol = _rel(dtf, dtf_o), _rel(dvol, dvol_o)
    print("%s full size, sampled rays: rel err tf %.2e params %.2e (of sum |block|) volume %.2e" %
          (name, e_tf, e_par, e_vol))
    assert np.linalg.norm(dtf_o) > 0 and np.linalg.norm(dvol_o) > 0
    assert e_tf <= TOL_GRAD and e_par <= TOL_GRAD and e_vol <= TOL_GRAD
    vr.free_volume(vid)


@pytest.mark.parametrize("kernel", [0, 3])
def test_uniform_gradients_optional(vr, torch, kernel):
    """dparams = NULL: the uniforms' gradient is not computed and (gamma = 0) the
    Hessian is not read; the transfer-function and voxel gradients are unchanged."""
    case = _cases()["head_1d_gamma0"]
    In32 = oracle.normalize(case["volume"]).astype(np.float32)
    vid = _setup(vr, torch, case, In32)
    n, H, W = case["cams"].shape[0], case["H"], case["W"]
    dl = torch.from_numpy(np.random.default_rng(76).normal(size=(n, H, W, 4)).astype(np.float32)).cuda()
    dtf, dpar, dvol = [x.cpu().numpy() for x in vr.render_backward(vid, case["cams"], W, H, dl, kernel=kernel)]
    dtf2, dpar2, dvol2 = vr.render_backward(vid, case["cams"], W, H, dl, kernel=kernel, want_params=False)
    assert dpar2 is None and np.abs(dpar).max() > 0
    np.testing.assert_allclose(dtf2.cpu().numpy(), dtf, rtol=1e-5, atol=1e-6 * np.abs(dtf).max())
    np.testing.assert_allclose(dvol2.cpu().numpy(), dvol, rtol=1e-5, atol=1e-6 * np.abs(dvol).max())
    vr.free_volume(vid)


def test_fit_checkpoint_resume_on_gpu(vr, torch, tmp_path):
    """The transfer-function fit through the C ABI, interrupted after a checkpoint and
    resumed from it, ends where the uninterrupted fit ends (float atomics in the
    backward make each run's gradients differ in the last bits, so within rounding)."""
    from paper_2605_19737_gb300 import autograd as ag
    from paper_2605_19737_gb300.fit import fit_transfer_function
    case = _cases()["head_1d"]
    In32 = oracle.normalize(case["volume"]).astype(np.float32)
    vid = _setup(vr, torch, case, In32)
    n, H, W = case["cams"].shape[0], case["H"], case["W"]
    fixed = {k: v for k, v in case["params"].items() if k not in ag.PARAM_NAMES}
    params = torch.tensor([case["params"][k] for k in ag.PARAM_NAMES], dtype=torch.float32)
    tf_target = np.clip(case["tf"] + np.random.default_rng(77).normal(0, 0.05, case["tf"].shape), 0, 1)
    with torch.no_grad():
        target = ag.render(vr, vid, torch.from_numpy(tf_target.astype(np.float32)).cuda(), params, case["cams"], W,
                           H, fixed)
    tf0 = torch.from_numpy(case["tf"]).cuda()
    ref_tf, ref_losses, _ = fit_transfer_function(vr, vid, case["cams"], W, H, tf0, target, fixed, params, steps=12)
    ck = str(tmp_path / "fit.pt")
    fit_transfer_function(vr, vid, case["cams"], W, H, tf0, target, fixed, params, steps=8, checkpoint=ck, every=4)
    tf, losses, _ = fit_transfer_function(vr, vid, case["cams"], W, H, tf0, target, fixed, params, steps=12,
                                          checkpoint=ck, every=4)
    assert len(losses) == 12 and losses[-1] < losses[0]
    np.testing.assert_allclose(losses, ref_losses, rtol=1e-4)
    np.testing.assert_allclose(tf.cpu().numpy(), ref_tf.cpu().numpy(), rtol=0, atol=1e-4)
    vr.free_volume(vid)
