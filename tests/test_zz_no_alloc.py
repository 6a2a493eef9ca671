"""GPU: the no-allocation batch entry point.

Some callers cannot allocate device memory at the moment they run the gather: an engine that
reserves its whole GPU budget up front and forbids allocations in its frame loop, or a plug-in
whose host application owns all device memory.  ssilvb_gather_batch_noalloc serves them with a
fixed scratch array inside the library.  Its results must equal ssilvb_gather_batch's, on two
calls in a row that share that array, and pass the oracle's parity gates; and a call must leave
the device's free memory unchanged.  Collected last on purpose."""
import numpy as np
import pytest

import scenegen
from scenegen import Params
from tests.gpu_util import check_tensors

pytestmark = pytest.mark.gpu


def _make(ctx, specs, keep=None):
    import torch

    import paper_2301_11376_gb300 as ssilvb
    noise = scenegen.ign_table()
    sh = scenegen.sh_environment(7)
    frames, hold = [], []
    for seed, W, H, kw in specs:
        g = scenegen.render(seed, W, H, 12, 4)
        prm = Params(**kw)
        d = torch.from_numpy(g.depth).cuda()
        n = torch.from_numpy(g.normal).cuda()
        r = torch.from_numpy(g.radiance).cuda()
        o0, o1, m = ssilvb.alloc_outputs(H, W, prm, "cuda", masks=True)
        a0, a1, am = ssilvb.alloc_outputs(H, W, prm, "cuda", masks=True)
        for t in (o0, a0):
            t.fill_(-5.0)
        f, keep = ctx.frame(d, n, r, g.camera, prm, o0, o1, m, noise=noise,
                            sh=sh if prm.ambient_cones else None, keep=keep)
        fa, keep = ctx.frame(d, n, r, g.camera, prm, a0, a1, am, noise=noise,
                             sh=sh if prm.ambient_cones else None, keep=keep)
        frames.append((f, fa))
        hold.append((g, d, n, r, (o0, o1, m), (a0, a1, am), prm))
    return frames, hold, keep


def _same(hold):
    for g, d, n, r, ours, theirs, prm in hold:
        for x, y in zip(ours, theirs):
            if x is None:
                continue
            if x.dtype.is_floating_point:
                assert float((x - y).abs().max()) <= 1e-6
            else:
                assert bool((x == y).all())


def _oracle(hold):
    noise, sh = scenegen.ign_table(), scenegen.sh_environment(7)
    for k, (g, d, n, r, (o0, o1, m), _, prm) in enumerate(hold):
        check_tensors(g, prm, noise, sh if prm.ambient_cones else None, o0, o1, m, seed=k)


SETS = [
    [(501, 96, 54, dict(num_slices=2, steps_per_side=8, thickness=0.2)),
     (502, 150, 97, dict(num_slices=4, steps_per_side=16, thickness=0.8, ambient_cones=4)),
     (503, 7, 3, dict(num_slices=1, steps_per_side=5))],
    [(511, 130, 66, dict(num_slices=3, steps_per_side=12, thickness=0.5, hit_rule=1)),
     (512, 64, 200, dict(num_slices=2, steps_per_side=24, thickness=0.3, thickness_slope=0.01))],
]


def test_noalloc_matches_batch_on_two_calls():
    import torch

    import paper_2301_11376_gb300 as ssilvb
    ssilvb.build()
    ctx = ssilvb.Context(0)
    made = [_make(ctx, specs) for specs in SETS]  # every device buffer exists before the calls
    # The first call on a device looks up the scratch array and may load the kernel's module: not
    # part of the measurement below.
    ssilvb.gather_batch_noalloc([f for f, _ in made[0][0]])
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for frames, hold, keep in made:  # two calls in a row through the same scratch array
        ssilvb.gather_batch_noalloc([f for f, _ in frames])
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before, "the call changed the device's free memory"
    for frames, hold, keep in made:
        ctx.gather_batch([fa for _, fa in frames])
    torch.cuda.synchronize()
    for frames, hold, keep in made:
        _same(hold)
        _oracle(hold)
    ctx.close()


def test_noalloc_rejects_more_than_its_limit():
    import paper_2301_11376_gb300 as ssilvb
    ssilvb.build()
    ctx = ssilvb.Context(0)
    frames, hold, keep = _make(ctx, [(520 + i, 8, 8, dict(num_slices=1, steps_per_side=2)) for i in range(17)])
    with pytest.raises(ssilvb.SsilvbError) as ei:
        ssilvb.gather_batch_noalloc([f for f, _ in frames])
    assert ei.value.code == 1 and "16" in str(ei.value)
    ctx.close()
