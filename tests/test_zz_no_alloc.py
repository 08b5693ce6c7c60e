"""The allocation-free walk entry point (for callers that must not allocate
device memory during a call) against the regular batched walk, through the C
ABI, on two calls in a row.  Collected last on purpose: it shares a fixed
device scratch array with nothing else, and a failure here leaves every other
test already run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2311_12818_gb300 import inputs as I  # noqa: E402


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_12818_gb300 import build, mpg
    build.build()
    return mpg


def _walk_both(M, ctx, wl, P):
    sc = M.Scene(ctx, wl)
    ref = M.Chains(wl)
    M.mpg_sample_seeds(ctx, sc, None, ref, P, wl.rng_seed, 0)
    na = M.Chains(wl)
    for name in ("x", "surf", "prim", "bary", "pdf", "status", "iters", "tau"):
        getattr(na, name).copy_(getattr(ref, name))
    M.mpg_manifold_walk(ctx, sc, ref, P)
    M.mpg_manifold_walk_noalloc(sc, na, P)
    torch.cuda.synchronize()
    return ref.aos(), na.aos()


@pytest.mark.parametrize("workload", ["mixed", "glass"])
def test_noalloc_walk_matches_batched_walk_on_two_calls(M, workload):
    ctx = M.Context(0)
    for call in range(2):
        if workload == "mixed":
            wl = I.mixed(nx=32, ny=16, spq=4, seed=0x4D50470004 + call)
            P = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True, k_uniform=0)
        else:
            wl = I.glass_sphere(n=24, spq=8, seed=0x4D50470002 + call)
            P = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, k_uniform=2)
        a, b = _walk_both(M, ctx, wl, P)
        ca, cb = a["status"] == 1, b["status"] == 1
        assert (a["status"] == b["status"]).mean() >= 0.999
        both = ca & cb
        assert both.sum() > 0.1 * wl.B
        for i in range(int(wl.k.max())):
            sel = both & (wl.k > i)
            if sel.any():
                d = np.linalg.norm(a["x"][sel, i] - b["x"][sel, i], axis=1)
                assert d.max() < 1e-4 * wl.scene_scale


def test_noalloc_rejects_batches_above_its_scratch(M):
    ctx = M.Context(0)
    wl = I.glass_sphere(n=256, spq=17)  # 1,114,112 chains > 1,048,576
    sc = M.Scene(ctx, wl)
    ch = M.Chains(wl)
    P = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, k_uniform=2)
    with pytest.raises(M.MpgError) as e:
        M.mpg_manifold_walk_noalloc(sc, ch, P)
    assert "at most" in str(e.value)
