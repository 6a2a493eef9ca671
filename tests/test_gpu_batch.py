"""GPU: the batched persistent launch over uneven frames equals per-frame gathers bit for bit,
and the autotuner's choices change no result; each batched frame also passes the oracle's parity
gates on its own (masks against the binary32 replica, outputs against FP64)."""
import math

import numpy as np
import pytest

import scenegen
from scenegen import Params
from tests.gpu_util import check_tensors, masks_to_u64, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    import paper_2301_11376_gb300 as ssilvb
    assert torch.cuda.is_available()
    ssilvb.build()
    c = ssilvb.Context(0)
    yield c
    c.close()


def _frames(ctx, specs, f16=False):
    """specs: (seed, W, H, params kwargs).  Returns (frames, keep, device outputs, gbuffers, params)."""
    import torch

    import paper_2301_11376_gb300 as ssilvb
    frames, outs, gbs, prms, keep = [], [], [], [], None
    noise = scenegen.ign_table()
    sh = scenegen.sh_environment(7)
    for seed, W, H, kw in specs:
        g = scenegen.render(seed, W, H, 12, 4)
        if f16:
            g = g.as_f16()
        prm = Params(**kw)
        d = torch.from_numpy(g.depth).cuda()
        n = torch.from_numpy(np.ascontiguousarray(g.normal)).cuda()
        r = torch.from_numpy(np.ascontiguousarray(g.radiance)).cuda()
        o0, o1, m = ssilvb.alloc_outputs(H, W, prm, "cuda", masks=True)
        o0.fill_(-3.0)
        f, keep = ctx.frame(d, n, r, g.camera, prm, o0, o1, m, noise=noise, sh=sh if prm.ambient_cones else None,
                            keep=keep)
        frames.append(f)
        outs.append((o0, o1, m, d, n, r))
        gbs.append(g)
        prms.append(prm)
    return frames, keep, outs, gbs, prms


def _check_against_single(ctx, outs, gbs, prms, oracle_check=True):
    noise = scenegen.ign_table()
    sh = scenegen.sh_environment(7)
    for k, ((o0, o1, m, *_), g, prm) in enumerate(zip(outs, gbs, prms)):
        if oracle_check:  # the batched outputs against the oracle, before the single-frame comparison
            check_tensors(g, prm, noise, sh if prm.ambient_cones else None, o0, o1, m, seed=k)
        ref = run_gpu(ctx, g, prm, noise, sh if prm.ambient_cones else None)
        got0 = o0.cpu().numpy().reshape(-1, 4).astype(np.float64)
        assert np.array_equal(got0, ref[0])
        if prm.ambient_cones:
            assert np.array_equal(o1.cpu().numpy().reshape(-1, 4).astype(np.float64), ref[1])
        assert np.array_equal(masks_to_u64(m, prm.sector_count), ref[2])


UNEVEN = [
    (101, 96, 54, dict(num_slices=1, steps_per_side=8, thickness=0.1)),
    (102, 200, 130, dict(num_slices=4, steps_per_side=32, thickness=1.0)),
    (103, 33, 7, dict(num_slices=2, steps_per_side=12, thickness=0.4, hit_rule=1)),
    (104, 130, 129, dict(num_slices=3, steps_per_side=20, thickness=0.7, ambient_cones=4)),
    (105, 1, 1, dict(num_slices=2, steps_per_side=8)),
    (106, 257, 64, dict(num_slices=4, steps_per_side=9, thickness=0.25, thickness_slope=0.02)),
]


@pytest.mark.parametrize("mode,rows,graph,order", [(1, 1, 1, 0), (1, 2, 2, 0), (1, 4, 1, 0), (1, 3, 2, 0), (2, 0, 0, 0),
                                                  (2, 0, 0, 2)])
def test_batch_equals_single(ctx, mode, rows, graph, order):
    import torch
    frames, keep, outs, gbs, prms = _frames(ctx, UNEVEN)
    ctx.set_tuning(rows_per_tile=rows, use_graph=graph, batch_mode=mode, block_order=order)
    ctx.gather_batch(frames)
    torch.cuda.synchronize()
    ctx.set_tuning()
    _check_against_single(ctx, outs, gbs, prms)


@pytest.mark.parametrize("nb", [64, 128])
def test_batch_fp16_wide_masks(ctx, nb):
    import torch
    specs = [(110 + i, 64 + 37 * i, 40 + 11 * i, dict(num_slices=1 + i % 4, steps_per_side=8 + 5 * i,
                                                     sector_count=nb, ambient_cones=8)) for i in range(5)]
    for mode in (1, 2):
        frames, keep, outs, gbs, prms = _frames(ctx, specs, f16=True)
        ctx.set_tuning(batch_mode=mode)
        ctx.gather_batch(frames)
        torch.cuda.synchronize()
        ctx.set_tuning()
        _check_against_single(ctx, outs, gbs, prms)


def test_batch_ring_reuse_and_many_in_flight(ctx):
    """More batches than the context's ring of in-flight slots, on two streams, then the cached
    graph of a slot reused for different frames."""
    import torch
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    all_sets = []
    for k in range(9):
        ctx.set_tuning(batch_mode=1 + k % 2)
        specs = [(200 + 10 * k + i, 48 + 16 * i, 32 + 8 * k, dict(num_slices=1 + (i + k) % 3, steps_per_side=6 + k))
                 for i in range(3)]
        frames, keep, outs, gbs, prms = _frames(ctx, specs)
        ctx.gather_batch(frames, stream=streams[k % 2])
        all_sets.append((keep, outs, gbs, prms))
    torch.cuda.synchronize()
    ctx.set_tuning()
    for keep, outs, gbs, prms in all_sets:
        _check_against_single(ctx, outs, gbs, prms)


def test_batch_rejects_mixed_kinds(ctx):
    import paper_2301_11376_gb300 as ssilvb
    specs = [(300, 32, 32, dict(sector_count=32)), (301, 32, 32, dict(sector_count=64))]
    frames, keep, outs, gbs, prms = _frames(ctx, specs)
    with pytest.raises(ssilvb.SsilvbError) as ei:
        ctx.gather_batch(frames)
    assert ei.value.code == 2
    specs = [(302, 32, 32, dict(thickness=0.5)), (303, 32, 32, dict(thickness=math.inf))]
    frames, keep, outs, gbs, prms = _frames(ctx, specs)
    with pytest.raises(ssilvb.SsilvbError):
        ctx.gather_batch(frames)


def test_autotune_keeps_results(ctx):
    import torch
    frames, keep, outs, gbs, prms = _frames(ctx, UNEVEN[:4])
    t = ctx.autotune(frames)
    assert t.occupancy in (8, 9) and t.rows_per_tile in (1, 2, 4) and t.use_graph in (1, 2)
    assert t.batch_mode in (1, 2)
    for o in outs:
        o[0].fill_(-3.0)
    ctx.gather_batch(frames)
    torch.cuda.synchronize()
    _check_against_single(ctx, outs, gbs, prms)
    one, keep1, outs1, gbs1, prms1 = _frames(ctx, UNEVEN[1:2])
    t1 = ctx.autotune(one)
    assert t1.mapping in (1, 2)
    _check_against_single(ctx, outs1, gbs1, prms1)


def test_batch_builtin_noise_equals_the_table(ctx):
    """Frames of one batch with the library's built-in noise (noise_mode 1) at different frame
    indices give the bits of single-frame gathers passed the same tables (noise_mode 2), and
    pass the oracle's gates."""
    import torch

    import paper_2301_11376_gb300 as ssilvb
    specs = [(130 + k, 72 + 16 * k, 40 + 8 * k, dict(num_slices=1 + k % 3, steps_per_side=6 + 3 * k)) for k in range(4)]
    frames, keep, hold = [], None, []
    for k, (seed, W, H, kw) in enumerate(specs):
        g = scenegen.render(seed, W, H, 12, 4)
        prm = Params(**kw)
        d = torch.from_numpy(g.depth).cuda()
        n = torch.from_numpy(g.normal).cuda()
        r = torch.from_numpy(g.radiance).cuda()
        o0, o1, m = ssilvb.alloc_outputs(H, W, prm, "cuda", masks=True)
        f, keep = ctx.frame(d, n, r, g.camera, prm, o0, o1, m, noise=("ign", 3 * k + 1), keep=keep)
        frames.append(f)
        hold.append((g, prm, o0, m, scenegen.ign_table(3 * k + 1), (d, n, r)))  # inputs stay alive
    ctx.gather_batch(frames)
    torch.cuda.synchronize()
    for g, prm, o0, m, table, _ in hold:
        ref = run_gpu(ctx, g, prm, table)
        assert np.array_equal(o0.cpu().numpy().reshape(-1, 4).astype(np.float64), ref[0])
        assert np.array_equal(masks_to_u64(m, prm.sector_count), ref[2])
        check_tensors(g, prm, table, None, o0, None, m)
