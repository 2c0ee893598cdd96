"""polypic_p2g_noalloc: P2G on the library's built-in scratch, for callers that
cannot allocate device memory while they run.  Its grids must match
polypic_p2g's (which uses a caller workspace) within the parity tolerance, on
two calls in a row (the second call finds the first call's leftovers in the
shared built-in array).  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2308_01060_gb300 import polypic as pp
from paper_2308_01060_gb300 import scenes
from gpu_util import np_, rel, sorted_particles

TOL = 1e-5


@pytest.mark.gpu
@pytest.mark.parametrize("R,fmt", [(27, "f32"), (8, "f32")])
def test_noalloc_p2g_matches_workspace_p2g_twice(R, fmt):
    sc = scenes.parity_scene(n=32, R=R, seed=31, random_mode_init=True)
    ctx = pp.Context(sc.n, sc.dx, R, coeff_format=fmt)
    ps, ws = sorted_particles(ctx, sc.fluid)
    ref = ctx.new_grid(vel=False)
    pp.polypic_p2g(ctx, ps, ref, ws)
    for _ in range(2):
        g = ctx.new_grid(vel=False)
        for a in range(3):
            g.mass[a].fill_(3.0)
            g.mom[a].fill_(3.0)
        pp.polypic_p2g_noalloc(ctx, ps, g)
        for a in range(3):
            assert rel(np_(g.mass[a]), np_(ref.mass[a])) <= TOL
            assert rel(np_(g.mom[a]), np_(ref.mom[a])) <= TOL
    assert pp.polypic_check_device_status(ctx) == 0


@pytest.mark.gpu
def test_noalloc_p2g_rejects_grids_beyond_its_scratch():
    ctx = pp.Context((128, 128, 128), 1 / 128, 4)          # 8192 tiles > 2048
    ps = ctx.new_particles(0)
    g = ctx.new_grid(vel=False)
    with pytest.raises(pp.PolyPICError) as ei:
        pp.polypic_p2g_noalloc(ctx, ps, g)
    assert ei.value.name == "WORKSPACE"
