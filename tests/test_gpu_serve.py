"""GPU: the continuous-batching server gives every request the same result as a gather of
that request alone (bit for bit), while batches overlap on the device."""
import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu


def test_serving_results_equal_alone():
    import torch

    import paper_2301_11376_gb300 as ssilvb
    from paper_2301_11376_gb300 import serve
    ssilvb.build()
    ctx = ssilvb.Context(0)
    pool = serve.ResidentPool()
    sizes = [(160, 90), (320, 180), (256, 144), (480, 270)]
    keys = []
    for i, (W, H) in enumerate(sizes):
        pool.add(("s", i), scenegen.render(700 + i, W, H, 16, 4))
        keys.append(("s", i))
    reqs = serve.poisson_requests(42, 64, 2e-5, keys, None, nd_range=(1, 8), nb_choices=(32, 64),
                                  ns_choices=(8, 16))
    got = {}

    def keep(req, o0, o1):
        got[req.rid] = o0.clone()

    srv = serve.Server(ctx, pool, arena_bytes=64 << 20, max_inflight=4, max_batch=8)
    st = srv.run(reqs, on_done=keep)
    torch.cuda.synchronize()
    assert st.served == len(reqs) and st.dropped == 0
    assert st.max_inflight_seen >= 2  # batches overlapped on the device
    for req in reqs:
        d, n, r, cam = pool.items[req.key]
        H, W = d.shape
        o0, _, _ = ssilvb.alloc_outputs(H, W, req.params, "cuda")
        ctx.gather(d, n, r, cam, req.params, o0, None, None, noise=req.noise)
        torch.cuda.synchronize()
        assert torch.equal(got[req.rid], o0), req.rid
    # the naive baseline serves the same results
    got_plain = {}
    plain = serve.PlainServer(ctx, pool)
    st2 = plain.run(reqs[:16], on_done=lambda req, o0, o1: got_plain.__setitem__(req.rid, o0.clone()))
    assert st2.served == 16
    for rid, v in got_plain.items():
        assert torch.equal(v, got[rid])
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
