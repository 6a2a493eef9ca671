"""GPU: multi-bounce (Section 4.3) — the next frame's light buffer is direct + gain * GI.
Gain 0 reproduces the single bounce; iterating frames through the light buffer raises GI
monotonically and converges for a gain below the feedback limit."""
import numpy as np
import pytest

import oracle
import scenegen
from scenegen import Params

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


def _run(ctx, d, n, r, cam, prm, noise, light=True, direct=None):
    import torch

    import paper_2301_11376_gb300 as ssilvb
    H, W = d.shape
    o0, _, _ = ssilvb.alloc_outputs(H, W, prm, "cuda")
    lo = torch.full_like(r, -1.0) if light else None
    ctx.gather(d, n, r, cam, prm, o0, None, None, noise=noise, light_out=lo, direct=direct)
    torch.cuda.synchronize()
    return o0, lo


@pytest.mark.parametrize("f16", [False, True])
def test_gain_zero_is_single_bounce(ctx, f16):
    import torch
    g = scenegen.render(801, 96, 64, 12, 4)
    if f16:
        g = g.as_f16()
    noise = scenegen.ign_table()
    d, n, r = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (g.depth, g.normal, g.radiance))
    prm = Params(num_slices=3, steps_per_side=10, bounce_gain=0.0)
    o_plain, _ = _run(ctx, d, n, r, g.camera, prm, noise, light=False)
    o_mb, lo = _run(ctx, d, n, r, g.camera, prm, noise)
    assert torch.equal(o_plain, o_mb)
    ref = r.clone()
    ref[..., 3] = 0
    assert torch.equal(lo, ref)


@pytest.mark.parametrize("f16", [False, True])
def test_light_buffer_is_direct_plus_gain_gi(ctx, f16):
    import torch
    g = scenegen.render(802, 80, 60, 12, 4)
    if f16:
        g = g.as_f16()
    noise = scenegen.ign_table()
    gain = 0.6
    d, n, r = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (g.depth, g.normal, g.radiance))
    prm = Params(num_slices=2, steps_per_side=12, bounce_gain=gain)
    o0, lo = _run(ctx, d, n, r, g.camera, prm, noise)
    gi = o0.cpu().numpy()[..., :3].astype(np.float64)
    direct = g.radiance[..., :3].astype(np.float64)
    expect = (np.float32(gain) * gi + direct).astype(np.float32)
    if f16:
        expect = expect.astype(np.float16)
    got = lo.cpu().numpy()[..., :3]
    np.testing.assert_allclose(got.astype(np.float64), expect.astype(np.float64), rtol=0, atol=1e-3 if f16 else 1e-6)
    # against the FP64 oracle's indirect light
    e0 = oracle.fp64(oracle.Problem(g, prm, noise))[0]
    exp64 = gain * e0[:, :3].reshape(got.shape) + direct
    assert np.abs(got.astype(np.float64) - exp64).max() < (2e-3 if f16 else 1e-4)


def test_bounces_increase_and_converge(ctx):
    import torch
    g = scenegen.render(803, 96, 72, 16, 6)
    noise = scenegen.ign_table()
    d, n, r = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (g.depth, g.normal, g.radiance))
    prm = Params(num_slices=4, steps_per_side=12, radius=3.0, bounce_gain=0.5)
    light = r
    gis = []
    for _ in range(5):  # each frame: this frame's direct light r, last frame's light buffer as input
        o0, lo = _run(ctx, d, n, light, g.camera, prm, noise, direct=r)
        gis.append(o0[..., :3].clone())
        light = lo
    assert float(gis[0].max()) > 0.0
    for a, b in zip(gis, gis[1:]):
        assert bool((b >= a - 1e-6).all())
    inc = [float((b - a).max()) for a, b in zip(gis, gis[1:])]
    # GI_{k+1} - GI_k = gain * W (GI_k - GI_{k-1}) with row sums of W <= 1: geometric decay
    for a, b in zip(inc, inc[1:]):
        assert b <= 0.5 * a + 1e-6
