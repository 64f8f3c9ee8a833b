"""Host-side tiling rules of the Lorenz-96 sweeps (eda_plan_tiling: no GPU).

A sweep tile must cover its owned points plus a halo on each side that is
wider than the distance an error from outside travels over K RK4 steps
(8 points per tangent-linear step, 11 per adjoint step: the reach
tests/test_tile_halo.py measures with the oracle's steps), fit the thread
and shared-memory limits of one CTA, and the CTAs of a vector must cover n.
"""
import itertools

import pytest

import paper_2605_23571_gb300 as P

SMEM_LIMIT = 227 * 1024


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.build()


@pytest.mark.parametrize("fp64", [True, False])
def test_cluster_plans_cover_the_state_with_the_halo(fp64):
    runs = (2, 4) if fp64 else (2, 4, 8)
    seen = 0
    for n, cs, K, C, w in itertools.product((40, 97, 300, 997, 4096, 30000), range(1, 17), (1, 2, 4, 8, 16),
                                            (0,) + runs, (2, 50)):
        p = P.plan_tiling(n, fp64, w, "cluster", cs=cs, K=K, C=C)
        if p is None:
            continue
        seen += 1
        assert p["kind"] == "cluster" and p["ctas_per_vector"] == cs and p["K"] == K
        assert p["C"] == (C if C else (4 if fp64 else 8)) and p["C"] in runs
        assert p["halo"] == 8 * K + 8                                   # > 8K + 3, the K-step reach
        assert p["threads"] % 32 == 0 and 32 <= p["threads"] <= 512
        assert cs * p["owned"] >= n and (cs - 1) * p["owned"] < n       # every CTA owns points
        assert p["owned"] + 2 * p["halo"] <= p["threads"] * p["C"]      # tile + both halos in registers
        assert p["threads"] * p["C"] - (p["owned"] + 2 * p["halo"]) < 32 * p["C"]  # no idle warp
        assert 0 < p["smem"] <= SMEM_LIMIT
    assert seen > 100


@pytest.mark.parametrize("fp64", [True, False])
def test_multi_launch_tiles(fp64):
    for n, K, threads in itertools.product((30000, 65536, 100000), (1, 4, 8, 16), (0, 128, 256)):
        p = P.plan_tiling(n, fp64, 50, "multi-launch", threads=threads, K=K)
        if p is None:
            continue
        A = threads if threads else (512 if fp64 else 256)
        assert p["kind"] == "multi-launch" and p["threads"] == A and p["C"] == (4 if fp64 else 8)
        assert p["halo"] == 8 * K + 8
        assert p["owned"] == A * p["C"] - 2 * p["halo"] and p["owned"] >= 64
        assert p["ctas_per_vector"] == -(-n // p["owned"])
        assert p["smem"] <= SMEM_LIMIT
    assert P.plan_tiling(65536, False, 50, "multi-launch", K=8, C=8) is None   # run length is fixed


@pytest.mark.parametrize("fp64", [True, False])
def test_warp_plans(fp64):
    runs = (2, 4) if fp64 else (4, 8)
    seen = 0
    for n, cs, K, C in itertools.product((1000, 2048, 4096), (2, 3, 5, 8, 16), (4, 8, 16), runs):
        p = P.plan_tiling(n, fp64, 50, "warp", cs=cs, K=K, C=C)
        if p is None:
            continue
        seen += 1
        hw = -(-11 // C) * C                                             # warp halo: the adjoint's reach
        lw = 32 * C - 2 * hw                                             # points a warp owns
        warps = p["threads"] // 32
        assert p["threads"] % 32 == 0 and p["threads"] <= 512 and lw > 0
        assert warps * lw >= p["owned"] + 2 * p["halo"] and warps * lw <= n   # distinct points per CTA
        assert cs * p["owned"] >= n and p["halo"] == 8 * K + 8
        assert p["smem"] <= SMEM_LIMIT
    assert seen > 10


def test_impossible_shapes_are_refused():
    assert P.plan_tiling(4096, False, 50, "cluster", cs=5, K=8, C=16) is None   # FP32 runs are 2, 4 or 8
    assert P.plan_tiling(4096, True, 50, "cluster", cs=5, K=8, C=8) is None     # FP64 runs are 2 or 4
    assert P.plan_tiling(4096, False, 50, "cluster", cs=1, K=8, C=4) is None    # one CTA cannot hold it
    assert P.plan_tiling(4096, False, 50, "cluster", cs=17, K=8) is None        # cluster limit 16
    assert P.plan_tiling(0, False, 50, "cluster", cs=1, K=8) is None


@pytest.mark.parametrize("kind", ["cluster", "multi-launch", "warp"])
def test_refresh_period_is_bounded(kind):
    # the halo 8K + 8 is an int: an absurd K is refused instead of wrapping
    kw = {"cs": 5} if kind != "multi-launch" else {}
    C = 0 if kind != "warp" else 8
    for K in (4097, 1 << 28, (1 << 31) - 1):
        assert P.plan_tiling(4096, False, 50, kind, K=K, C=C, **kw) is None


@pytest.mark.parametrize("fp64", [True, False])
def test_checkpointed_multi_launch_plans(fp64):
    # the halo covers the recomputed states' edge errors plus the adjoint's
    # reach (19K + 8), and K states of the region fit in shared memory
    for K in (1, 2, 4, 6, 8):
        p = P.plan_tiling(65536, fp64, 50, "multi-launch", K=K, ckpt=True)
        assert p is not None and p["halo"] == 19 * K + 8 and p["K"] == K
        assert p["owned"] == p["threads"] * p["C"] - 2 * p["halo"] and p["owned"] >= 64
        assert p["smem"] <= SMEM_LIMIT
        assert p["smem"] >= K * p["threads"] * p["C"] * (8 if fp64 else 4)
    # too long a segment for shared memory (FP64) or for the tile
    assert P.plan_tiling(65536, True, 50, "multi-launch", K=20, ckpt=True) is None
