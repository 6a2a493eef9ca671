"""GPU: the interleaved F16X8 storage (normal and radiance in one 16-byte record per pixel) gives
the same bits as the two F16X4 planes it holds (same binary16 values), on every entry point that
reads a G-buffer, and passes the oracle's gates; invalid F16X8 arguments enqueue nothing."""
import math

import numpy as np
import pytest

import scenegen
from scenegen import Params
from tests.gpu_util import check_tensors, masks_to_u64

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


def _both(ctx, g, prm, noise, sh):
    """Planar and interleaved device gathers of one FP16 G-buffer: (out0, out1, masks) for each."""
    import torch

    import paper_2301_11376_gb300 as ssilvb
    H, W = g.depth.shape
    d = torch.from_numpy(g.depth).cuda()
    n = torch.from_numpy(g.normal).cuda()
    r = torch.from_numpy(g.radiance).cuda()
    nr = torch.from_numpy(g.interleaved_f16()).cuda()
    res = []
    for normal, radiance in ((n, r), (nr, None)):
        o0, o1, m = ssilvb.alloc_outputs(H, W, prm, "cuda", masks=True)
        o0.fill_(-9.0)
        ctx.gather(d, normal, radiance, g.camera, prm, o0, o1, m, noise=noise, sh=sh)
        res.append((o0, o1, m))
    torch.cuda.synchronize()
    return res


def _equal(a, b):
    import torch
    for x, y in zip(a, b):
        if x is not None:
            assert torch.equal(x, y)


@pytest.mark.parametrize("W,H,seed,kw", [
    (96, 64, 41, dict(num_slices=3, steps_per_side=12, ambient_cones=4)),
    (61, 47, 42, dict(num_slices=2, steps_per_side=20, sector_count=64, step_mode=1, ambient_cones=8)),
    (45, 37, 43, dict(num_slices=4, steps_per_side=9, sector_count=128, thickness=math.inf, hit_rule=1)),
    (33, 7, 44, dict(num_slices=1, steps_per_side=5, thickness_slope=0.05)),
])
def test_interleaved_equals_planar_and_passes_parity(ctx, W, H, seed, kw):
    g = scenegen.render(seed, W, H, 10, 3).as_f16()
    prm = Params(**kw)
    noise, sh = scenegen.ign_table(), scenegen.sh_environment(7) if prm.ambient_cones else None
    planar, inter = _both(ctx, g, prm, noise, sh)
    _equal(planar, inter)
    check_tensors(g, prm, noise, sh, *inter, min_agree=0.95)


@pytest.mark.parametrize("nb", [32, 64])
def test_interleaved_4k_workload_equals_planar(ctx, nb):
    w = scenegen.workload_4k(sector_count=nb)
    planar, inter = _both(ctx, w.gbuf, w.params, w.noise, w.sh)
    _equal(planar, inter)


def test_interleaved_host_buffers_and_batch(ctx):
    import torch

    import paper_2301_11376_gb300 as ssilvb
    g = scenegen.render(45, 300, 530, 16, 4).as_f16()  # 530 rows: two host row bands
    prm = Params(num_slices=2, steps_per_side=10, ambient_cones=2)
    noise, sh = scenegen.ign_table(), scenegen.sh_environment(7)
    H, W = g.depth.shape
    planar, _ = _both(ctx, g, prm, noise, sh)
    ref = [t.cpu().numpy() if t is not None else None for t in planar]
    # host buffers, synchronous and pipelined
    nr = g.interleaved_f16()
    for asynchronous in (False, True):
        o0 = np.full((H, W, 4), -9.0, np.float32)
        o1 = np.full((H, W, 4), -9.0, np.float32)
        m = np.zeros((prm.num_slices, H, W, 1), np.int32)
        ctx.gather_host(g.depth, nr, None, g.camera, prm, o0, o1, m, noise=noise, sh=sh, asynchronous=asynchronous)
        ctx.synchronize()
        assert np.array_equal(o0, ref[0]) and np.array_equal(o1, ref[1]) and np.array_equal(m, ref[2])
    # a batch of interleaved frames (both launch forms); a batch mixing layouts is refused (the
    # storage format is a property of the kernel variant, like the sector count)
    d = torch.from_numpy(g.depth).cuda()
    n = torch.from_numpy(g.normal).cuda()
    r = torch.from_numpy(g.radiance).cuda()
    nrd = torch.from_numpy(nr).cuda()
    outs, frames, keep = [], [], None
    for _ in range(3):
        o0, o1, m = ssilvb.alloc_outputs(H, W, prm, "cuda", masks=True)
        f, keep = ctx.frame(d, nrd, None, g.camera, prm, o0, o1, m, noise=noise, sh=sh, keep=keep)
        frames.append(f)
        outs.append((o0, o1, m))
    for mode in (1, 2):
        ctx.set_tuning(batch_mode=mode)
        ctx.gather_batch(frames)
        torch.cuda.synchronize()
        for o in outs:
            _equal(planar, o)
    ctx.set_tuning()
    mixed, keep = ctx.frame(d, n, r, g.camera, prm, *outs[0], noise=noise, sh=sh, keep=keep)
    with pytest.raises(ssilvb.SsilvbError) as ei:
        ctx.gather_batch([frames[0], mixed])
    assert ei.value.code == 2


def test_interleaved_invalid_arguments(ctx):
    import ctypes

    import torch

    import paper_2301_11376_gb300 as ssilvb
    g = scenegen.render(46, 32, 32, 4, 1).as_f16()
    d = torch.from_numpy(g.depth).cuda()
    nr = torch.from_numpy(g.interleaved_f16()).cuda()
    other = nr.clone()
    out0 = torch.full((32, 32, 4), 5.0, device="cuda")
    keep = ssilvb._HostArrays()
    pc = ssilvb._params_c(Params(), keep)
    cam = ssilvb._camera_c(g.camera)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    o = ssilvb.Output(out0.data_ptr(), 512, None, 0, None, None, 0)
    cases = [
        # radiance must be the normal plane itself
        (ssilvb.Gbuffer(32, 32, d.data_ptr(), 128, nr.data_ptr(), 512, 2, other.data_ptr(), 512, 2, None, 0), o, 1),
        # pitch below 16 bytes per pixel
        (ssilvb.Gbuffer(32, 32, d.data_ptr(), 128, nr.data_ptr(), 256, 2, nr.data_ptr(), 256, 2, None, 0), o, 1),
        # interleaved normal with planar radiance format
        (ssilvb.Gbuffer(32, 32, d.data_ptr(), 128, nr.data_ptr(), 512, 2, nr.data_ptr(), 512, 1, None, 0), o, 2),
        # no multi-bounce light buffer with the interleaved layout
        (ssilvb.Gbuffer(32, 32, d.data_ptr(), 128, nr.data_ptr(), 512, 2, nr.data_ptr(), 512, 2, None, 0),
         ssilvb.Output(out0.data_ptr(), 512, None, 0, None, other.data_ptr(), 512), 2),
    ]
    for gb, oo, code in cases:
        rc = ctx.lib.ssilvb_gather(ctx.handle, ctypes.byref(gb), ctypes.byref(cam), ctypes.byref(pc),
                                   ctypes.byref(oo), s)
        assert rc == code
    torch.cuda.synchronize()
    assert torch.all(out0 == 5.0)
