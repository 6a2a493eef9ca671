"""GPU: the continuous-batching server gives every request the same result as a gather of
that request alone (bit for bit), while batches overlap on the device, and every served result
passes the oracle's parity gates (outputs against FP64 on sampled pixels)."""
import dataclasses
import math

import numpy as np
import pytest

import scenegen
from tests.gpu_util import check_tensors

pytestmark = pytest.mark.gpu


def test_serving_results_equal_alone():
    import torch

    import paper_2301_11376_gb300 as ssilvb
    from paper_2301_11376_gb300 import serve
    ssilvb.build()
    ctx = ssilvb.Context(0)
    pool = serve.ResidentPool()
    sizes = [(160, 90), (320, 180), (256, 144), (480, 270)]
    keys, host = [], {}
    for i, (W, H) in enumerate(sizes):
        g = scenegen.render(700 + i, W, H, 16, 4)
        pool.add(("s", i), g)
        keys.append(("s", i))
        host[("s", i)] = g
    reqs = serve.poisson_requests(42, 64, 2e-5, keys, None, nd_range=(1, 8), nb_choices=(32, 64),
                                  ns_choices=(8, 16))
    # mixed kinds in one stream: batches group requests by what a batch call must share
    for q in reqs:
        if q.rid % 5 == 1:
            q.params = dataclasses.replace(q.params, thickness=math.inf)
        if q.rid % 7 == 2:
            q.params = dataclasses.replace(q.params, step_mode=1)
    got, got_masks = {}, {}

    def keep(req, o0, o1, masks):
        got[req.rid] = o0.clone()
        got_masks[req.rid] = masks.clone()

    srv = serve.Server(ctx, pool, arena_bytes=96 << 20, max_inflight=4, max_batch=8, with_masks=True)
    st = srv.run(reqs, on_done=keep)
    torch.cuda.synchronize()
    assert st.served == len(reqs) and st.dropped == 0
    assert st.max_inflight_seen >= 2  # batches overlapped on the device
    assert srv.arena.free == [(0, srv.arena.size)]  # every output block came back
    for req in reqs:
        d, n, r, cam = pool.items[req.key]
        H, W = d.shape
        o0, _, m = ssilvb.alloc_outputs(H, W, req.params, "cuda", masks=True)
        ctx.gather(d, n, r, cam, req.params, o0, None, m, noise=req.noise)
        torch.cuda.synchronize()
        assert torch.equal(got[req.rid], o0), req.rid
        assert torch.equal(got_masks[req.rid], m), req.rid  # masks bit-exact alone and in the mix
        # the served result against the oracle: masks against the replica, outputs against FP64
        check_tensors(host[req.key], req.params, req.noise, None, got[req.rid], None, got_masks[req.rid],
                      n_sample=3000, seed=req.rid, min_clear=0.5)  # up to 8 slices: fewer pixels clear in every slice
    # the naive baseline serves the same results
    got_plain = {}
    plain = serve.PlainServer(ctx, pool)
    st2 = plain.run(reqs[:16], on_done=lambda req, o0, o1: got_plain.__setitem__(req.rid, o0.clone()))
    assert st2.served == 16
    for rid, v in got_plain.items():
        assert torch.equal(v, got[rid])
    ctx.close()


def test_latency_budget_sheds_and_serves_the_rest_correctly():
    """Under a stream far above capacity with a latency budget, the server sheds at arrival and
    every request it serves still equals the same request alone."""
    import torch

    import paper_2301_11376_gb300 as ssilvb
    from paper_2301_11376_gb300 import serve
    ssilvb.build()
    ctx = ssilvb.Context(0)
    pool = serve.ResidentPool()
    keys = []
    for i, (W, H) in enumerate([(1280, 720), (1920, 1080)]):
        pool.add(("b", i), scenegen.render(720 + i, W, H, 16, 4))
        keys.append(("b", i))
    reqs = serve.poisson_requests(43, 300, 1e-5, keys, None, nd_range=(4, 8), nb_choices=(32, 64),
                                  ns_choices=(16, 32))
    got = {}
    srv = serve.Server(ctx, pool, arena_bytes=256 << 20, max_inflight=4, max_batch=8, budget_ms=20.0, rate=4e11)
    st = srv.run(reqs, on_done=lambda req, o0, o1: got.__setitem__(req.rid, o0.clone()))
    torch.cuda.synchronize()
    assert st.dropped > 0 and st.served == len(reqs) - st.dropped and st.served > 0
    assert st.within_budget <= st.served
    for req in reqs:
        if req.rid not in got:
            continue
        d, n, r, cam = pool.items[req.key]
        H, W = d.shape
        o0, _, _ = ssilvb.alloc_outputs(H, W, req.params, "cuda")
        ctx.gather(d, n, r, cam, req.params, o0, None, None, noise=req.noise)
        torch.cuda.synchronize()
        assert torch.equal(got[req.rid], o0), req.rid
    ctx.close()


def test_serving_interleaved_and_planar_pools():
    """Resident G-buffers in both FP16 layouts (two planes, and one interleaved F16X8 plane) served in
    one stream: batches never mix layouts, and each result equals the same request alone."""
    import torch

    import paper_2301_11376_gb300 as ssilvb
    from paper_2301_11376_gb300 import serve
    ssilvb.build()
    ctx = ssilvb.Context(0)
    pool = serve.ResidentPool()
    keys = []
    for i, (W, H) in enumerate([(200, 120), (320, 180)]):
        g = scenegen.render(740 + i, W, H, 16, 4).as_f16()
        pool.add(("p", i), g)
        pool.add(("i", i), g, interleaved=True)
        keys += [("p", i), ("i", i)]
    reqs = serve.poisson_requests(44, 40, 1e-5, keys, None, nd_range=(1, 4), nb_choices=(32, 64), ns_choices=(8,))
    got = {}
    srv = serve.Server(ctx, pool, arena_bytes=64 << 20, max_inflight=4, max_batch=8)
    st = srv.run(reqs, on_done=lambda req, o0, o1: got.__setitem__(req.rid, o0.clone()))
    torch.cuda.synchronize()
    assert st.served == len(reqs)
    for req in reqs:
        d, n, r, cam = pool.items[req.key]
        H, W = d.shape
        o0, _, _ = ssilvb.alloc_outputs(H, W, req.params, "cuda")
        ctx.gather(d, n, r, cam, req.params, o0, None, None, noise=req.noise)
        torch.cuda.synchronize()
        assert torch.equal(got[req.rid], o0), req.rid
    # the same request from the planar and the interleaved copy of a scene gives the same bits
    twin = {}
    for req in reqs:
        twin.setdefault((req.key[1], req.params.num_slices, req.params.sector_count, req.params.steps_per_side),
                        {})[req.key[0]] = got[req.rid]
    pairs = [v for v in twin.values() if len(v) == 2]
    for v in pairs:
        assert torch.equal(v["p"], v["i"])
    ctx.close()


def test_arena_first_fit():
    from paper_2301_11376_gb300 import serve
    pytest.importorskip("torch")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs CUDA")
    a = serve.OutputArena(4096)
    x = a.alloc(1000)
    y = a.alloc(1000)
    z = a.alloc(3000)
    assert x == (0, 1024) and y == (1024, 1024) and z is None
    a.release(*x)
    assert a.alloc(1024) == (0, 1024)
    a.release(0, 1024)
    a.release(*y)
    assert a.free == [(0, 4096)]
