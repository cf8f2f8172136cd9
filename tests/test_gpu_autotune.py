"""The launch-shape autotuner (to_autotune): it times every distinct z-chunk
length of the column-streaming operators on the context's grid and keeps
the fastest.  Chunking changes only which element layer a block recomputes,
never the order in which a node sums its element contributions, so every
operator gives bitwise the same result before and after tuning; and a
second context of the same grid takes the tuned shapes from the process
cache without timing."""

import numpy as np
import pytest

from gpu_helpers import Ctx, dev, host
from workloads import rand_density, rand_vector, small_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_autotune_keeps_results_and_caches(precision):
    from paper_2205_00385_gb300 import binding as B
    p = small_problem("cantilever3d", nelx=64, nely=32, nelz=40, mg_levels=4)
    rho0 = rand_density(p.nel, 71, 0.05, 1.0)
    rho1 = np.clip(rho0 + rand_density(p.nel, 72, -0.1, 0.1), 0.0, 1.0)
    x = dev(rand_vector(p.ndof, 73, fixed=p.fixed))
    r = dev(rand_vector(p.ndof, 74, fixed=p.fixed))

    def products(c):
        out = []
        for prec in (B.TO_PREC_NATIVE, B.TO_PREC_DF, B.TO_PREC_FP32, B.TO_PREC_FP64):
            for op in (B.TO_OP_K, B.TO_OP_DK):
                y = dev(np.zeros(p.ndof))
                B.to_apply(c.ctx, op, prec, x, y)
                out.append(host(y).copy())
        z = dev(np.zeros(p.ndof))
        B.to_vcycle(c.ctx, r, z)
        out.append(host(z).copy())
        u = dev(np.zeros(p.ndof))
        it, _, ok = B.to_mgcg_solve(c.ctx, 1e-8, 200, 0, u)
        out.append(host(u).copy())
        return out, it

    with Ctx(p, precision=precision) as c:
        c.set_density(rho0)
        c.set_density(rho1)
        before, it0 = products(c)
        res = B.to_autotune(c.ctx, reps=3)
        after, it1 = products(c)
    kinds = {q["kernel"] for q in res}
    assert {"op_apply", "op_resid", "op_smooth", "gal1_resid", "gal1_smooth"} <= kinds
    assert ("acc_apply" in kinds) == (precision == "mixed")
    for q in res:
        print(f"[autotune {precision}] {q}")
        assert q["candidates"] >= 3
        assert q["chosen_us"] <= q["heuristic_us"] * 1.0001
        assert q["chunk_layers"] == 0 or 2 <= q["chunk_layers"] <= p.nelz + 1
    assert it0 == it1
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    # a second context of the same grid takes the shapes from the cache
    with Ctx(p, precision=precision) as c2:
        c2.set_density(rho1)
        res2 = B.to_autotune(c2.ctx, reps=3)
    assert [q["candidates"] for q in res2] == [0] * len(res2)
    assert [q["chunk_layers"] for q in res2] == [q["chunk_layers"] for q in res]


def test_tall_tiles_give_the_same_bits():
    """The 16-row tile variant of the float32 finest-grid operator
    (TO_OPERATOR_TALL_TILES) computes every node's sum in the same order as
    the 8-row one: products, V-cycles and solves are bitwise the same, on a
    grid whose rows split unevenly into both tile heights."""
    from paper_2205_00385_gb300 import binding as B
    p = small_problem("cantilever3d", nelx=64, nely=40, nelz=24, mg_levels=4)
    rho = rand_density(p.nel, 75, 0.05, 1.0)
    x = dev(rand_vector(p.ndof, 76, fixed=p.fixed))
    r = dev(rand_vector(p.ndof, 77, fixed=p.fixed))
    out = []
    with Ctx(p, precision="mixed") as c:
        c.set_density(rho)
        for flags in (0, B.TO_OPERATOR_TALL_TILES):
            B.to_operator_options(c.ctx, flags)
            y = dev(np.zeros(p.ndof))
            B.to_apply(c.ctx, B.TO_OP_K, B.TO_PREC_FP32, x, y)
            z = dev(np.zeros(p.ndof))
            B.to_vcycle(c.ctx, r, z)
            u = dev(np.zeros(p.ndof))
            it, _, _ = B.to_mgcg_solve(c.ctx, 1e-8, 200, 0, u)
            out.append((host(y), host(z), host(u), it))
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)
    assert out[0][3] == out[1][3]


@pytest.mark.parametrize("tall", [False, True])
def test_work_list_launch_gives_the_same_bits(tall):
    """The work-list launch of the float32 finest-grid operator
    (TO_OPERATOR_WORK_LIST: one CTA per resident slot taking (tile, z-chunk)
    items from a counter) computes each item as the one-block-per-item
    launch does: products, V-cycles (captured graphs included, whose
    replays reuse the counters) and whole solves are bitwise the same, on a
    grid with more items than resident CTAs and on one with fewer."""
    from paper_2205_00385_gb300 import binding as B
    base = B.TO_OPERATOR_TALL_TILES if tall else 0
    for kw, levels in ((dict(nelx=64, nely=40, nelz=24), 4), (dict(nelx=16, nely=8, nelz=8), 2)):
        p = small_problem("cantilever3d", mg_levels=levels, **kw)
        rho = rand_density(p.nel, 78, 0.05, 1.0)
        x = dev(rand_vector(p.ndof, 79, fixed=p.fixed))
        r = dev(rand_vector(p.ndof, 80, fixed=p.fixed))
        out = []
        with Ctx(p, precision="mixed") as c:
            c.set_density(rho)
            for flags in (base, base | B.TO_OPERATOR_WORK_LIST):
                B.to_operator_options(c.ctx, flags)
                res = []
                for _ in range(2):   # the second call reuses the reset counters
                    y = dev(np.zeros(p.ndof))
                    B.to_apply(c.ctx, B.TO_OP_K, B.TO_PREC_FP32, x, y)
                    z = dev(np.zeros(p.ndof))
                    B.to_vcycle(c.ctx, r, z)
                    res += [host(y), host(z)]
                u = dev(np.zeros(p.ndof))
                it, _, _ = B.to_mgcg_solve(c.ctx, 1e-8, 200, 0, u)
                out.append((res, host(u), it))
        for a, b in zip(out[0][0], out[1][0]):
            assert np.array_equal(a, b)
        assert np.array_equal(out[0][1], out[1][1])
        assert out[0][2] == out[1][2] and out[0][2] > 0
