"""GPU parity: the CUDA gather (through the C ABI) against the CPU oracle.

Bitmasks must equal the binary32 replica's bit for bit; AO, GI and ambient must be
within 1e-4 of the FP64 oracle (Algorithm 1; Sections 3.1-3.3).
"""
import math

import numpy as np
import pytest

import oracle
import scenegen
from scenegen import Params
from tests.gpu_util import check_parity, run_gpu, sample_pixels, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    import paper_2301_11376_gb300 as ssilvb
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    ssilvb.build()
    c = ssilvb.Context(0)
    yield c
    c.close()


def test_256_full_frame(ctx):
    w = scenegen.workload_256()
    res = run_gpu(ctx, w.gbuf, w.params, w.noise)
    info = check_parity(w.gbuf, w.params, w.noise, None, res)
    assert info["agree"] > 0.999


SMALL = [
    # (W, H, seed, params kwargs, noise)
    (1, 1, 3, dict(num_slices=2, steps_per_side=4), True),
    (3, 5, 3, dict(num_slices=3, steps_per_side=5), True),
    (37, 29, 4, dict(num_slices=16, steps_per_side=3, radius=4.0), True),
    (61, 47, 5, dict(num_slices=1, steps_per_side=64, radius=3.0), True),
    (50, 40, 6, dict(num_slices=4, steps_per_side=8, thickness=math.inf), True),
    (50, 40, 7, dict(num_slices=4, steps_per_side=8, hit_rule=1), True),
    (64, 48, 8, dict(num_slices=3, steps_per_side=8, sector_count=64, ambient_cones=8), True),
    (64, 48, 9, dict(num_slices=2, steps_per_side=12, step_mode=1), True),
    (64, 48, 10, dict(num_slices=2, steps_per_side=8, thickness=0.1, thickness_slope=0.05), True),
    (64, 48, 11, dict(num_slices=2, steps_per_side=8, gi=False, ambient_cones=2), True),
    (64, 48, 12, dict(num_slices=2, steps_per_side=8, ambient_cones=1), False),
    (70, 33, 13, dict(num_slices=5, steps_per_side=7, sector_count=64, thickness=math.inf, hit_rule=1), True),
    (33, 70, 14, dict(num_slices=4, steps_per_side=10, sector_count=64, step_mode=1, ambient_cones=4), True),
    (64, 48, 15, dict(num_slices=3, steps_per_side=12, sector_count=128, ambient_cones=8), True),
    (45, 37, 16, dict(num_slices=2, steps_per_side=9, sector_count=128, thickness=math.inf, hit_rule=1), True),
    (50, 41, 17, dict(num_slices=5, steps_per_side=7, sector_count=128, step_mode=1, thickness_slope=0.03), True),
    (40, 30, 18, dict(num_slices=2, steps_per_side=1), True),                  # one step: a pair's second half idle
    (40, 30, 19, dict(num_slices=2, steps_per_side=6, radius=1e6), True),      # projected radius at its 2^20 cap
    (40, 30, 20, dict(num_slices=2, steps_per_side=6, radius=1e-4), True),     # every step on the centre pixel
    # small radius on a larger frame: the unchecked prefix loop covers whole sides; odd N_s leaves its last
    # pair's second step idle
    (200, 150, 23, dict(num_slices=3, steps_per_side=7, radius=0.5), True),
    (201, 149, 24, dict(num_slices=2, steps_per_side=9, radius=0.4, step_mode=1, sector_count=64), True),
    # most sides leave the screen part-way: each warp's unchecked prefix, then the checked steps
    (320, 180, 27, dict(num_slices=2, steps_per_side=24, radius=3.0), True),
    (320, 180, 28, dict(num_slices=2, steps_per_side=23, radius=3.0, step_mode=1, sector_count=128), True),
    # the largest width and height the ABI accepts, each with a handful of pixels across
    (16384, 5, 25, dict(num_slices=2, steps_per_side=6), True),
    (6, 16384, 26, dict(num_slices=2, steps_per_side=6, sector_count=64, ambient_cones=2), True),
]


@pytest.mark.parametrize("W,H,seed,kw,use_noise", SMALL)
def test_small_and_ragged(ctx, W, H, seed, kw, use_noise):
    g = scenegen.render(seed, W, H, 8, 3)
    prm = Params(**kw)
    noise = scenegen.ign_table() if use_noise else None
    sh = scenegen.sh_environment(7) if prm.ambient_cones else None
    res = run_gpu(ctx, g, prm, noise, sh)
    check_parity(g, prm, noise, sh, res, min_agree=0.95)


@pytest.mark.parametrize("f16", [False, True])
def test_fp16_storage(ctx, f16):
    g = scenegen.render(15, 80, 60, 8, 3)
    if f16:
        g = g.as_f16()
    prm = Params(num_slices=3, steps_per_side=10, ambient_cones=4)
    noise, sh = scenegen.ign_table(), scenegen.sh_environment(7)
    res = run_gpu(ctx, g, prm, noise, sh)
    check_parity(g, prm, noise, sh, res)


@pytest.mark.parametrize("W,H,nb", [(150, 77, 32), (333, 1100, 32), (333, 1100, 64), (97, 1601, 128)])
def test_block_orders_bit_identical(ctx, W, H, nb):
    """The class-mapped blocks in raster order of patches or in bands of about 32 patch rows (the
    order the library picks for frames of 2^22 pixels or more, forced here on small frames): the
    same patches, so identical bits.  1100 and 1601 rows give 69 and 101 patch rows: three bands of
    23, and four of 26 with the last one three rows short (its blocks past the frame exit); a ragged
    right edge (333, 97 pixels) leaves part of the last patch column empty.  An unknown order is
    rejected."""
    g = scenegen.render(31, W, H, 10, 4)
    prm = Params(num_slices=2, steps_per_side=7, sector_count=nb, ambient_cones=2)
    noise, sh = scenegen.ign_table(), scenegen.sh_environment(7)
    results = []
    try:
        for order in (1, 2, 0):
            ctx.set_tuning(block_order=order)
            results.append(run_gpu(ctx, g, prm, noise, sh))
        with pytest.raises(Exception, match="block_order"):
            ctx.set_tuning(block_order=3)
    finally:
        ctx.set_tuning()
    for r in results[1:]:
        for a, b in zip(results[0], r):
            assert np.array_equal(a, b)
    check_parity(g, prm, noise, sh, results[0], pixels=sample_pixels(H, W, 20000, 5))


@pytest.mark.parametrize("nb,step_mode,f16", [(32, 0, True), (64, 1, False), (128, 0, False)])
def test_launch_choices_bit_identical(ctx, nb, step_mode, f16):
    """Every single-frame launch choice (class-strided warps with the 8- or 9-block register
    budget, natural 32x8 tiles) computes the same binary32 sequence: identical bits."""
    g = scenegen.render(22, 150, 77, 8, 3)
    if f16:
        g = g.as_f16()
    prm = Params(num_slices=3, steps_per_side=9, sector_count=nb, step_mode=step_mode, ambient_cones=4)
    noise, sh = scenegen.ign_table(), scenegen.sh_environment(7)
    results = []
    try:
        for mapping, occupancy in ((2, 8), (2, 9), (1, 0)):
            ctx.set_tuning(mapping=mapping, occupancy=occupancy)
            results.append(run_gpu(ctx, g, prm, noise, sh))
    finally:
        ctx.set_tuning()
    for r in results[1:]:
        for a, b in zip(results[0], r):
            assert np.array_equal(a, b)
    check_parity(g, prm, noise, sh, results[0])


def test_pitched_inputs(ctx):
    g = scenegen.render(16, 45, 31, 8, 3)
    prm = Params(num_slices=2, steps_per_side=6)
    noise = scenegen.ign_table()
    a = run_gpu(ctx, g, prm, noise, pad=0)
    b = run_gpu(ctx, g, prm, noise, pad=11)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    check_parity(g, prm, noise, None, b)


def test_sky_only_frame(ctx):
    g = scenegen.render(17, 40, 30, 0, 0)
    g.depth[:] = np.inf
    prm = Params(num_slices=2, steps_per_side=4, ambient_cones=4)
    sh = scenegen.sh_environment(7)
    o0, o1, m = run_gpu(ctx, g, prm, None, sh)
    assert np.all(o0 == [0, 0, 0, 1]) and np.all(o1 == 0) and np.all(m == 0)


def test_flat_plane_exact(ctx):
    g = scenegen.hand_plane(41, 33, normal_view=(0.5, -0.3, 0.81), point_depth=6.0)
    prm = Params(num_slices=4, steps_per_side=7, radius=2.0, thickness=0.5)
    o0, _, m = run_gpu(ctx, g, prm, None)
    assert np.all(m == 0) and np.all(o0[:, 3] == 1.0) and np.all(o0[:, :3] == 0.0)


def test_deterministic_and_stream(ctx):
    import torch
    g = scenegen.render(18, 64, 64, 8, 3)
    prm = Params(num_slices=4, steps_per_side=8)
    noise = scenegen.ign_table()
    s = torch.cuda.Stream()
    a = run_gpu(ctx, g, prm, noise, stream=s)
    b = run_gpu(ctx, g, prm, noise)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    import ctypes
    assert ctx.lib.ssilvb_get_status(ctx.handle, ctypes.c_void_p(s.cuda_stream)) == 0


def test_1080p_full_masks_and_sampled_fp64(ctx):
    w = scenegen.workload_1080p()
    res = run_gpu(ctx, w.gbuf, w.params, w.noise)
    H, W = w.gbuf.depth.shape
    # masks of every pixel against the replica
    prob = oracle.Problem(w.gbuf, w.params, w.noise)
    _, _, rm = oracle.fp32(prob)
    assert np.array_equal(res[2], rm)
    check_parity(w.gbuf, w.params, w.noise, None, res, pixels=sample_pixels(H, W, 20000, 1))


@pytest.mark.parametrize("nb", [32, 64, 128])
def test_4k_precision_form_sampled(ctx, nb):
    """The benchmark workload at full size and launch configuration, checked on sampled pixels:
    FP32 depth with FP16 normal/radiance, 4 slices, 32 steps, 4 ambient cones."""
    w = scenegen.workload_4k(sector_count=nb)
    res = run_gpu(ctx, w.gbuf, w.params, w.noise, w.sh)
    H, W = w.gbuf.depth.shape
    info = check_parity(w.gbuf, w.params, w.noise, w.sh, res, pixels=sample_pixels(H, W, 12000, 2))
    assert info["agree"] > 0.98


@pytest.mark.parametrize("nb", [32, 64, 128])
def test_4k_full_frame_every_pixel(ctx, nb):
    """The benchmark workload in full, every gate on every pixel: all 8.29 M x 4 slice masks
    bit-exact against the binary32 replica, every pixel's AO, GI and ambient within 1e-4 of the
    decision-forced FP64 evaluation and within 1e-6 of the replica, the free-running FP64 oracle
    matched wherever decisions are clear of rounding, every mask flip explained."""
    w = scenegen.workload_4k(sector_count=nb)
    res = run_gpu(ctx, w.gbuf, w.params, w.noise, w.sh)
    info = check_parity(w.gbuf, w.params, w.noise, w.sh, res)
    assert info["n"] == 3840 * 2160 and info["agree"] > 0.999


def test_maximum_frame_sampled(ctx):
    """The largest frame the ABI accepts, 16384 x 16384 (2^28 pixels: the largest grid, pixel
    coordinates and mask offsets), FP16 normal/radiance, ambient cones and the masks of every
    slice; checked on sampled pixels (corners, edge midpoints and uniform draws), gathered on the
    device so that no full-frame array crosses to the host."""
    import torch

    import paper_2301_11376_gb300 as ssilvb
    N = 16384
    g = scenegen.render(31, N, N, 64, 16).as_f16()
    prm = Params(num_slices=2, steps_per_side=8, ambient_cones=2)
    noise, sh = scenegen.ign_table(), scenegen.sh_environment(7)
    d, n, r = to_device(g)
    out0, out1, m = ssilvb.alloc_outputs(N, N, prm, "cuda", masks=True)
    out0.fill_(-7.0)
    ctx.gather(d, n, r, g.camera, prm, out0, out1, m, noise=noise, sh=sh)
    torch.cuda.synchronize()
    del d, n, r
    xy = sample_pixels(N, N, 3000, 6)
    idx = torch.from_numpy(xy[:, 1].astype(np.int64) * N + xy[:, 0]).cuda()
    o0 = out0.view(-1, 4)[idx].cpu().numpy().astype(np.float64)
    o1 = out1.view(-1, 4)[idx].cpu().numpy().astype(np.float64)
    mk = m.view(prm.num_slices, -1)[:, idx].cpu().numpy().view(np.uint32).T.astype(np.uint64)
    del out0, out1, m
    torch.cuda.empty_cache()
    info = check_parity(g, prm, noise, sh, (o0, o1, mk), pixels=xy, gathered=True)
    assert info["agree"] > 0.98


def test_empty_and_oversized_frames_rejected(ctx):
    """Frames with no rows or no columns, and frames wider or taller than 16384 pixels, are
    rejected before any launch (INVALID_ARG) and leave the outputs untouched."""
    import torch

    import paper_2301_11376_gb300 as ssilvb
    cam = scenegen.Camera(16.0, 16.0, 16.0, 16.0)
    for H, W in [(0, 32), (32, 0), (1, 16385), (16385, 1)]:
        d = torch.ones((H, W), device="cuda")
        n = torch.zeros((H, W, 4), device="cuda")
        r = torch.zeros((H, W, 4), device="cuda")
        out0 = torch.full((H, W, 4), 5.0, device="cuda")
        with pytest.raises(ssilvb.SsilvbError) as ei:
            ctx.gather(d, n, r, cam, Params(), out0, None, None)
        assert ei.value.code == 1
        torch.cuda.synchronize()
        assert torch.all(out0 == 5.0)


def test_host_buffers_equal_device_buffers(ctx):
    import torch

    import paper_2301_11376_gb300 as ssilvb
    g = scenegen.render(19, 72, 40, 8, 3).as_f16()
    prm = Params(num_slices=2, steps_per_side=8, ambient_cones=4)
    noise, sh = scenegen.ign_table(), scenegen.sh_environment(7)
    a = run_gpu(ctx, g, prm, noise, sh)
    H, W = g.depth.shape
    o0 = np.zeros((H, W, 4), np.float32)
    o1 = np.zeros((H, W, 4), np.float32)
    m = np.zeros((prm.num_slices, H, W), np.uint32)
    ctx.gather_host(g.depth, g.normal, g.radiance, g.camera, prm, o0, o1, m, noise=noise, sh=sh)
    assert np.array_equal(o0.reshape(-1, 4), a[0].astype(np.float32))
    assert np.array_equal(o1.reshape(-1, 4), a[1].astype(np.float32))
    assert np.array_equal(m.reshape(prm.num_slices, -1).T.astype(np.uint64), a[2])
    del torch, ssilvb


@pytest.mark.parametrize("f16", [False, True])
def test_host_buffers_in_row_bands(ctx, f16):
    """Host-buffer calls on frames of 512+ rows run as row-band launches whose outputs are copied
    back while later bands compute: uneven bands, masks of every slice, ambient output and the
    multi-bounce light buffer must equal the single device launch bit for bit."""
    import torch
    g = scenegen.render(21, 96, 1037, 8, 3)
    if f16:
        g = g.as_f16()
    prm = Params(num_slices=3, steps_per_side=8, sector_count=64, ambient_cones=4, bounce_gain=0.7)
    noise, sh = scenegen.ign_table(), scenegen.sh_environment(7)
    H, W = g.depth.shape
    direct = np.ascontiguousarray((g.radiance * 0.5).astype(g.radiance.dtype))
    # the device launch
    d, n, r = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (g.depth, g.normal, g.radiance))
    dd = torch.from_numpy(direct).cuda()
    import paper_2301_11376_gb300 as ssilvb
    do0, do1, dm = ssilvb.alloc_outputs(H, W, prm, "cuda", masks=True)
    dlo = torch.zeros_like(r)
    ctx.gather(d, n, r, g.camera, prm, do0, do1, dm, noise=noise, sh=sh, light_out=dlo, direct=dd)
    torch.cuda.synchronize()
    # the same frame through host buffers
    o0 = np.zeros((H, W, 4), np.float32)
    o1 = np.zeros((H, W, 4), np.float32)
    m = np.zeros((prm.num_slices, H, W), np.uint64)
    lo = np.zeros_like(g.radiance)
    ctx.gather_host(g.depth, g.normal, g.radiance, g.camera, prm, o0, o1, m, noise=noise, sh=sh,
                    light_out=lo, direct=direct)
    assert np.array_equal(o0, do0.cpu().numpy())
    assert np.array_equal(o1, do1.cpu().numpy())
    assert np.array_equal(m.view(np.int32).reshape(-1), dm.cpu().numpy().reshape(-1))  # [N_d][H][W] u64 words
    assert np.array_equal(lo, dlo.cpu().numpy())
    assert np.abs(lo[..., :3].astype(np.float64)).max() > 0


def test_host_buffers_asynchronous_stream_of_frames(ctx):
    """ssilvb_gather_host_async: frames of growing size enqueued back to back (two staging lanes,
    one frame's copies overlapping the next frame's gather, staging grown between uses) equal the
    synchronous call frame by frame, bit for bit, also when synchronous calls are interleaved."""
    prm = Params(num_slices=2, steps_per_side=8, sector_count=64, ambient_cones=4)
    noise, sh = scenegen.ign_table(), scenegen.sh_environment(7)
    frames = [scenegen.render(40 + k, 64 + 16 * k, 520 + 40 * k, 8, 3) for k in range(5)]

    def outputs(g):
        H, W = g.depth.shape
        return (np.zeros((H, W, 4), np.float32), np.zeros((H, W, 4), np.float32),
                np.zeros((prm.num_slices, H, W), np.uint64))

    expected = []
    for g in frames:
        o = outputs(g)
        ctx.gather_host(g.depth, g.normal, g.radiance, g.camera, prm, *o, noise=noise, sh=sh)
        expected.append(o)
    got = [outputs(g) for g in frames]
    for k, (g, o) in enumerate(zip(frames, got)):
        if k == 2:  # a synchronous call in the middle of the stream
            ctx.gather_host(g.depth, g.normal, g.radiance, g.camera, prm, *o, noise=noise, sh=sh)
        else:
            ctx.gather_host(g.depth, g.normal, g.radiance, g.camera, prm, *o, noise=noise, sh=sh, asynchronous=True)
    ctx.synchronize()
    for k, (a, b) in enumerate(zip(expected, got)):
        for x, y in zip(a, b):
            assert np.array_equal(x, y), k


def test_invalid_arguments_enqueue_nothing(ctx):
    import torch

    import paper_2301_11376_gb300 as ssilvb
    g = scenegen.render(20, 32, 32, 4, 1)
    d = torch.from_numpy(g.depth).cuda()
    n = torch.from_numpy(g.normal).cuda()
    r = torch.from_numpy(g.radiance).cuda()
    out0 = torch.full((32, 32, 4), 5.0, device="cuda")
    bad = [Params(num_slices=0), Params(num_slices=17), Params(steps_per_side=65), Params(radius=-1.0),
           Params(thickness=0.0), Params(sector_count=48), Params(sector_count=96), Params(hit_rule=2),
           Params(ambient_cones=3)]
    for prm in bad:
        with pytest.raises(ssilvb.SsilvbError) as ei:
            ctx.gather(d, n, r, g.camera, prm, out0, None, None)
        assert ei.value.code == 1
    with pytest.raises(ssilvb.SsilvbError) as ei:
        ctx.gather(d, n.half(), r, g.camera, Params(), out0, None, None)
    assert ei.value.code == 2
    # a host pointer where device memory is required
    with pytest.raises(ssilvb.SsilvbError):
        ctx.gather(torch.from_numpy(g.depth), n, r, g.camera, Params(), out0, None, None)
    # misaligned planes and pitches
    big = torch.zeros(32 * 33 + 1, device="cuda")
    with pytest.raises(ssilvb.SsilvbError) as ei:
        ctx.gather(big[1:32 * 32 + 1].view(32, 32), n, r, g.camera, Params(), out0, None, None)
    assert ei.value.code == 1
    short = torch.zeros(32 * 30 * 4 + 8 * 4, device="cuda").as_strided((32, 32, 4), (30 * 4, 4, 1))
    with pytest.raises(ssilvb.SsilvbError) as ei:  # out0 pitch shorter than a row of the image
        ctx.gather(d, n, r, g.camera, Params(), short, None, None)
    assert ei.value.code == 1
    torch.cuda.synchronize()
    assert torch.all(out0 == 5.0)


@pytest.mark.parametrize("frame", [1, 7, 63])
def test_temporal_noise_frames(ctx, frame):
    """Per-frame noise rotation (Section 3.1: the integral is distributed spatially and
    temporally): each frame's table is an input like any other and the gather stays exact."""
    g = scenegen.render(30 + frame, 72, 56, 10, 3)
    prm = Params(num_slices=2, steps_per_side=10, step_mode=1)
    noise = scenegen.ign_table(frame)
    res = run_gpu(ctx, g, prm, noise)
    check_parity(g, prm, noise, None, res)


@pytest.mark.parametrize("frame", [0, 5, 63, 64, 200])
def test_builtin_noise_table_equals_the_ign_input(ctx, frame):
    """noise_mode 1: the library's own 4x4 interleaved-gradient table (Section 3.1 "directions with
    random offset"; Section 4.3 temporal jitter) gives the same bits as passing the same table
    (computed independently on the host) as noise_mode 2, and passes the parity gates."""
    g = scenegen.render(40 + frame % 7, 72, 56, 10, 3)
    prm = Params(num_slices=2, steps_per_side=10, sector_count=64, step_mode=frame % 2)
    a = run_gpu(ctx, g, prm, ("ign", frame))
    table = scenegen.ign_table(frame)
    b = run_gpu(ctx, g, prm, table)
    for x, y in zip(a, b):
        if x is not None:
            assert np.array_equal(x, y)
    check_parity(g, prm, table, None, a, min_agree=0.95)


def test_noise_mode_arguments_checked(ctx):
    import ctypes

    import torch

    import paper_2301_11376_gb300 as ssilvb
    g = scenegen.render(21, 32, 32, 4, 1)
    d = torch.from_numpy(g.depth).cuda()
    n = torch.from_numpy(g.normal).cuda()
    r = torch.from_numpy(g.radiance).cuda()
    out0 = torch.full((32, 32, 4), 5.0, device="cuda")
    with pytest.raises(ssilvb.SsilvbError) as ei:
        ctx.gather(d, n, r, g.camera, Params(), out0, None, None, noise=("ign", -1))
    assert ei.value.code == 1
    keep = ssilvb._HostArrays()
    table = scenegen.ign_table()
    gb = ssilvb.Gbuffer(32, 32, d.data_ptr(), 128, n.data_ptr(), 512, 0, r.data_ptr(), 512, 0, None, 0)
    o = ssilvb.Output(out0.data_ptr(), 512, None, 0, None, None, 0)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for mode, with_table in [(3, False), (-1, False), (2, False), (0, True), (1, True)]:
        pc = ssilvb._params_c(Params(), keep, table if with_table else None)
        pc.noise_mode = mode
        if not with_table:
            pc.noise_table = None
        rc = ctx.lib.ssilvb_gather(ctx.handle, ctypes.byref(gb), ctypes.byref(ssilvb._camera_c(g.camera)),
                                   ctypes.byref(pc), ctypes.byref(o), s)
        assert rc == 1, (mode, with_table)
    torch.cuda.synchronize()
    assert torch.all(out0 == 5.0)
