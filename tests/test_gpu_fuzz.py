"""GPU parity on seeded random problems (tests/fuzz_cases.py): random sizes from 1x1 up, every
parameter of the ABI in random combination (N_d 1-16, N_s 1-64, N_b 32/64/128, both hit rules,
both step modes, finite and infinite thickness, thickness slope, 0-8 ambient cones, GI on/off),
FP32 or FP16 storage, no noise / the built-in table / a random table, and camera intrinsics and
view rotation perturbed away from the scene generator's symmetric camera, the patches in raster
or band order.  Every gate of check_parity on every pixel, through the C ABI."""
import math

import pytest

from tests.fuzz_cases import case
from tests.gpu_util import check_parity, run_gpu

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


@pytest.mark.parametrize("k", range(40))
def test_random_problem(ctx, k):
    g, prm, noise, table, sh = case(k)
    # odd cases run the class-mapped patches in bands (the order of large frames), even ones in
    # raster order: both orders over the random sizes
    ctx.set_tuning(block_order=1 + k % 2)
    try:
        res = run_gpu(ctx, g, prm, noise, sh)
    finally:
        ctx.set_tuning()
    # The agreement and clear-pixel floors only guard against a vacuous comparison; random slice
    # counts up to 16 make fully clear pixels rarer.  The floor/ceil rule with infinite thickness puts
    # every sample in the tangent plane of a flat surface on a rounding boundary (its run ends on the
    # hemisphere edge, where floor/ceil is discontinuous), so there FP64 and binary32 flip a sector on
    # a large share of pixels and the mean difference from the free-running FP64 oracle (G4) exceeds
    # 1e-4; G3 explains every flip and G2 (FP64 on the binary32 decisions) holds on every pixel.
    boundary_heavy = prm.hit_rule == 1 and math.isinf(prm.thickness)
    check_parity(g, prm, table, sh, res, min_agree=0.3 if boundary_heavy else 0.9, min_clear=0.0,
                 mean_gate=not boundary_heavy)
