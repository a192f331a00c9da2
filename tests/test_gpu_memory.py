"""Device-memory accounting, the per-context memory cap and the out-of-memory paths.

Allocation failures are made on the host (vr_debug_fail_alloc, vr_set_memory_limit):
the library sees cudaErrorMemoryAllocation from its own allocator and must return
VR_ERR_OOM, leak nothing, and leave the context and its volumes usable. Nothing here
faults the GPU."""

import numpy as np
import pytest

from phantoms import workloads
from tests.gpu_util import assert_rgba_parity, oracle_render_case, torch_cuda

pytestmark = pytest.mark.gpu

SIGMAS = (1.0, 2.0)


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def case():
    c = workloads.scaled_brainweb((40, 48, 36), width=48, height=36, n_cams=2)
    c["params"] = dict(c["params"], tf_mode=0)
    c["tf"] = c["tf"][:1]  # 1D table: the first row of the 2D one
    return c


def _is_oom(err):
    import paper_2605_19737_gb300 as pkg
    from paper_2605_19737_gb300.vr import VR_ERR_OOM
    return isinstance(err, pkg.VRError) and err.status == VR_ERR_OOM


def _steps(vr, torch, case, state):
    """The API calls of one render + backward + batch cycle, each as (name, fn)."""
    W, H, cams = case["W"], case["H"], case["cams"]

    def load():
        state["vid"] = vr.load_volume(case["volume"], case["spacing"])  # host data: staged copy

    def precompute():
        vr.precompute_morphology(state["vid"], SIGMAS)

    def params():
        vr.set_tissue_params(state["vid"], case["tf"], **case["params"])

    def render():
        state["img"] = vr.render(state["vid"], cams, W, H).cpu().numpy()

    def backward():
        g = torch.ones((cams.shape[0], H, W, 4), dtype=torch.float32, device="cuda")
        dtf, dpar, dvol = vr.render_backward(state["vid"], cams, W, H, g, want_volume=True)
        state["grad"] = (dtf.cpu().numpy(), dpar.cpu().numpy(), dvol.cpu().numpy())

    def batch():
        outs = [torch.zeros((H, W, 4), dtype=torch.float32, device="cuda") for _ in range(cams.shape[0])]
        state["bid"] = vr.batch_create([(state["vid"], cams[i], outs[i], W, H) for i in range(cams.shape[0])])
        vr.batch_render(state["bid"])
        torch.cuda.synchronize()
        state["batch"] = np.stack([o.cpu().numpy() for o in outs])

    return [("load", load), ("precompute", precompute), ("params", params), ("render", render),
            ("backward", backward), ("batch", batch)]


def _cleanup(vr, state):
    if "bid" in state:
        vr.batch_free(state.pop("bid"))
    if "vid" in state:
        vr.free_volume(state.pop("vid"))


def test_memory_used_counts_library_buffers(torch, case):
    import paper_2605_19737_gb300 as pkg
    vr = pkg.Context(0)
    try:
        base = vr.memory_used()
        assert 0 < base <= 4096  # the context's status/work words
        state = {}
        for _, fn in _steps(vr, torch, case, state)[:3]:
            fn()
        nz, ny, nx = case["volume"].shape
        nb = [(n - 1 + 7) // 8 for n in (nx, ny, nz)]
        nbricks = nb[0] * nb[1] * nb[2]
        nvox = nx * ny * nz
        held = vr.memory_used() - base
        # at least: normalised volume, intensity bricks (12^3 floats), derived bricks
        # (9^3 x 12 floats), vesselness volume and bricks
        assert held >= 4 * nvox * 2 + 6912 * nbricks * 2 + 34992 * nbricks
        vr.free_volume(state.pop("vid"))
        scratch = vr.memory_used() - base
        # what stays is scratch the context reuses (staging copy, vesselness scratch)
        assert scratch < held
        for _, fn in _steps(vr, torch, case, state)[:3]:
            fn()
        vr.free_volume(state.pop("vid"))
        assert vr.memory_used() - base == scratch  # no growth on a second cycle
    finally:
        vr.close()


def test_injected_allocation_failures(torch, case):
    """Fail the n-th allocation of a cycle on a fresh context, for every n: the call
    that needed it raises VR_ERR_OOM (or, for the optional derived bricks, falls back
    to the per-sample stencils); repeating the failed call and the rest of the cycle
    gives the clean results; after freeing, the context holds no more than after a
    clean cycle."""
    import paper_2605_19737_gb300 as pkg
    from paper_2605_19737_gb300.vr import VR_ERR_NOT_READY
    vr = pkg.Context(0)
    clean = {}
    try:
        for _, fn in _steps(vr, torch, case, clean):
            fn()
        _cleanup(vr, clean)
        after_clean = vr.memory_used()
    finally:
        vr.close()
    failures = []
    for n in range(64):
        vr = pkg.Context(0)
        try:
            state = {}
            steps = _steps(vr, torch, case, state)
            vr.debug_fail_alloc(n)
            failed = None
            for k, (name, fn) in enumerate(steps):
                try:
                    fn()
                except pkg.VRError as e:
                    assert _is_oom(e), "%s: %s" % (name, e)
                    failed = k
                    break
            pending = vr.debug_fail_alloc(-1)
            if failed is None and pending >= 0:
                _cleanup(vr, state)
                break  # the cycle makes fewer than n + 1 allocations
            if failed is None:
                # the injected failure hit the derived bricks: same images within rounding
                failures.append("derived")
                np.testing.assert_allclose(state["img"], clean["img"], rtol=0, atol=2e-4)
                np.testing.assert_array_equal(state["batch"], state["img"])
                _cleanup(vr, state)
                assert vr.memory_used() <= after_clean
                continue
            name = steps[failed][0]
            failures.append(name)
            if name == "load":
                assert "vid" not in state
                assert vr.memory_used() <= after_clean
            if name in ("precompute", "params"):
                # the volume is not renderable until the failed call is repeated
                with pytest.raises(pkg.VRError) as ei:
                    vr.render(state["vid"], case["cams"], case["W"], case["H"])
                assert ei.value.status == VR_ERR_NOT_READY
            for _, fn in steps[failed:]:
                fn()
            np.testing.assert_array_equal(state["img"], clean["img"])
            np.testing.assert_array_equal(state["batch"], clean["batch"])
            for a, b in zip(state["grad"], clean["grad"]):
                # float atomics: the summation order may differ between runs
                np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-5 * float(np.abs(b).max()))
            _cleanup(vr, state)
            assert vr.memory_used() <= after_clean, "leak after a failure in %s" % name
        finally:
            vr.close()
    else:
        pytest.fail("a cycle made more than 64 allocations")
    # every call of the cycle that allocates was made to fail at least once
    assert {"load", "precompute", "params", "backward", "batch", "derived"} <= set(failures), failures


def test_memory_limit(torch, case):
    """A cap below a volume's needs makes vr_load_volume fail with OOM (nothing held);
    a cap with room for everything but the derived bricks makes the precompute fall
    back to the per-sample stencils, whose image still matches the oracle."""
    import paper_2605_19737_gb300 as pkg
    vr = pkg.Context(0)
    try:
        base = vr.memory_used()
        vr.set_memory_limit(base + 4096)
        with pytest.raises(pkg.VRError) as ei:
            vr.load_volume(case["volume"], case["spacing"])
        assert _is_oom(ei.value)
        assert vr.memory_used() <= base + 4096
        # measure a full cycle without a cap, then allow it less the derived bricks
        vr.set_memory_limit(0)
        state = {}
        for _, fn in _steps(vr, torch, case, state)[:3]:
            fn()
        full = vr.memory_used()
        _cleanup(vr, state)
        nz, ny, nx = case["volume"].shape
        nbricks = np.prod([(n - 1 + 7) // 8 for n in (nx, ny, nz)])
        vr.set_memory_limit(full - 34992 * nbricks + 1024)
        steps = _steps(vr, torch, case, state)
        for _, fn in steps[:4]:
            fn()
        assert vr.memory_used() <= full - 34992 * nbricks + 1024
        res = oracle_render_case(case, brick_empty=vr.get_bricks(state["vid"])[1])
        assert_rgba_parity(state["img"], res, what="stencil fallback under a memory cap")
        _cleanup(vr, state)
    finally:
        vr.close()
