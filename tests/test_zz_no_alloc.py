"""The allocation-free walk entry point against the regular batched walk,
through the C ABI, on two calls in a row.

Some callers cannot allocate device memory during a call (a renderer whose
frame loop forbids cudaMalloc, a code whose device memory belongs to its own
pool allocator); mpg_manifold_walk_noalloc keeps its scratch in a fixed
device array inside the library for them.  Both entry points run the same
persistent walk kernels with the same schedule, so their outputs must be
identical bit for bit: a stale queue counter, bucket or chain order left in
the shared array by the previous call would show up as a difference.

Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test."""
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
    ctx.sync()
    M.mpg_manifold_walk_noalloc(sc, na, P)
    torch.cuda.synchronize()
    return ref, na


def _workload(M, name, call):
    if name.startswith("mixed"):
        wl = I.mixed(nx=32, ny=16, spq=4, seed=0x4D50470004 + call)
        sched = dict(walk_group=1) if name == "mixed_group" else {}
        return wl, M.params_from(wl.params, walk_mode=M.WALK_BATCHED, tau_random=True, k_uniform=0, **sched)
    if name == "glass_block64":
        wl = I.glass_sphere(n=24, spq=8, seed=0x4D50470002 + call)
        return wl, M.params_from(wl.params, walk_mode=M.WALK_BATCHED, block_threads=64, k_uniform=2)
    if name == "water":  # heightfield: every reprojection and seed runs the BVH traversal
        wl = I.water(n=48, spq=4, seed=0x4D50470003 + call)
        return wl, M.params_from(wl.params, walk_mode=M.WALK_BATCHED, k_uniform=0, ctas_per_sm=2)
    raise ValueError(name)


@pytest.mark.parametrize("name", ["mixed", "mixed_group", "glass_block64", "water"])
def test_noalloc_walk_is_bit_identical_to_batched_walk_on_two_calls(M, name):
    ctx = M.Context(0)
    for call in range(2):
        wl, P = _workload(M, name, call)
        ref, na = _walk_both(M, ctx, wl, P)
        for f in ("status", "iters", "x", "surf", "prim", "bary"):
            a, b = getattr(ref, f), getattr(na, f)
            assert torch.equal(a, b), (name, call, f, int((a != b).sum()))
        st = ref.status.cpu().numpy()
        assert (st == 1).sum() > 0.1 * wl.B
        assert not (st == 255).any()  # every seeded chain was walked


def test_noalloc_rejects_batches_above_its_scratch(M):
    ctx = M.Context(0)
    wl = I.glass_sphere(n=256, spq=17)  # 1,114,112 chains > 1,048,576
    sc = M.Scene(ctx, wl)
    ch = M.Chains(wl)
    P = M.params_from(wl.params, walk_mode=M.WALK_BATCHED, k_uniform=2)
    with pytest.raises(M.MpgError) as e:
        M.mpg_manifold_walk_noalloc(sc, ch, P)
    assert "at most" in str(e.value)
