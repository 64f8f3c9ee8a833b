"""eda_hvp_noalloc: the Hessian-vector products of eda_hvp for callers that
cannot allocate device memory while they run (for example a thread that is
capturing a CUDA graph in global mode, where cudaMalloc is illegal, or a
cycle confined to a preallocated memory budget).  Its scratch is a fixed
array inside the library, shared by every call; the products must equal
those of eda_hvp on two calls in a row (the second reusing the scratch the
first left behind).  Collected last so that a run stopping at the first
failure has run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

import eda_synth as S
from helpers import problem, rowrel

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_23571_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_hvp_matches_eda_hvp_on_two_calls(precision):
    import torch
    dev = torch.device("cuda:0")
    spec = S.spec_small(300, 16, 7, every_var=2, every_step=2, length_scale=6.0, seed=9)
    taps, xb, y = problem(spec)
    prec = P.EDA_FP64 if precision == "fp64" else P.EDA_MIXED
    with P.Handle.from_spec(spec, taps, precision=prec) as h:
        h.eda_set_trajectory(torch.tensor(xb, device=dev), torch.tensor(y, device=dev))
        cols = torch.tensor([3, 0, 6, 1, 1, 5], dtype=torch.int32, device=dev)
        assert cols.numel() * spec.p <= P.lib().eda_hvp_noalloc_capacity(1 if precision == "fp64" else 0)
        for call in range(2):
            V = torch.tensor(S.gaussian_matrix(cols.numel(), spec.n, 20 + call), device=dev)
            ref = torch.empty_like(V)
            out = torch.full_like(V, float("nan"))
            h.eda_hvp(cols, V, ref, True)
            h.eda_hvp_noalloc(cols, V, out, True)
            torch.cuda.synchronize()
            # the same sweep on the same inputs: equal to rounding
            assert rowrel(out.cpu().numpy(), ref.cpu().numpy()).max() < 1e-12
            # without the identity, on a different column set
            out2 = torch.empty_like(V[:3])
            ref2 = torch.empty_like(V[:3])
            h.eda_hvp(cols[:3].contiguous(), V[:3].contiguous(), ref2, False)
            h.eda_hvp_noalloc(cols[:3].contiguous(), V[:3].contiguous(), out2, False)
            torch.cuda.synchronize()
            assert rowrel(out2.cpu().numpy(), ref2.cpu().numpy()).max() < 1e-12


def test_noalloc_rejects_host_memory_and_oversized_batches():
    import torch
    dev = torch.device("cuda:0")
    spec = S.spec_small(64, 8, 3, every_var=1, every_step=1, length_scale=2.0, seed=2)
    taps, xb, y = problem(spec)
    with P.Handle.from_spec(spec, taps, precision=P.EDA_FP64) as h:
        h.eda_set_trajectory(xb, y)
        cols = torch.zeros(2, dtype=torch.int32, device=dev)
        V = torch.zeros(2, spec.n, dtype=torch.float64, device=dev)
        with pytest.raises(P.EdaError) as e:
            h.eda_hvp_noalloc(cols, V.cpu(), torch.zeros(2, spec.n, dtype=torch.float64), True)
        assert e.value.code == P.EDA_ERR_INVALID
        big = int(P.lib().eda_hvp_noalloc_capacity(1) // spec.p) + 1
        cb = torch.zeros(big, dtype=torch.int32, device=dev)
        Vb = torch.zeros(big, spec.n, dtype=torch.float64, device=dev)
        with pytest.raises(P.EdaError) as e:
            h.eda_hvp_noalloc(cb, Vb, torch.empty_like(Vb), True)
        assert e.value.code == P.EDA_ERR_INVALID
        assert "exceed" in str(e.value)


@pytest.mark.parametrize("entry", ["eda_hvp", "eda_hvp_noalloc"])
def test_member_index_out_of_range_gives_nan_rows(entry):
    # a device member_of_col is checked by the kernel: a bad index reads no
    # trajectory row and turns that column's output into NaN; the other
    # columns are computed as usual
    import torch
    dev = torch.device("cuda:0")
    spec = S.spec_small(300, 16, 4, every_var=2, every_step=2, length_scale=6.0, seed=9)
    taps, xb, y = problem(spec)
    with P.Handle.from_spec(spec, taps, precision=P.EDA_FP64) as h:
        h.eda_set_trajectory(torch.tensor(xb, device=dev), torch.tensor(y, device=dev))
        V = torch.tensor(S.gaussian_matrix(4, spec.n, 5), device=dev)
        good = torch.tensor([1, 2, 3, 0], dtype=torch.int32, device=dev)
        bad = torch.tensor([1, spec.n_members, 3, -1], dtype=torch.int32, device=dev)
        ref = torch.empty_like(V)
        out = torch.zeros_like(V)
        h.eda_hvp(good, V, ref, True)
        getattr(h, entry)(bad, V, out, True)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.isnan(o[1]).all() and np.isnan(o[3]).all()
        assert rowrel(o[[0, 2]], ref.cpu().numpy()[[0, 2]]).max() < 1e-12
        # a host member_of_col is checked before any work
        with pytest.raises(P.EdaError) as e:
            h.eda_hvp(bad.cpu().numpy(), V, out, True)
        assert e.value.code == P.EDA_ERR_INVALID


def test_noalloc_rejects_multi_launch_tilings():
    # multi-launch sweeps pass their state through buffers the handle
    # allocates, so the allocation-free entry point refuses them
    import torch
    from helpers import env
    dev = torch.device("cuda:0")
    spec = S.spec_small(600, 8, 3, every_var=2, every_step=2, length_scale=3.0, seed=3)
    taps, xb, y = problem(spec)
    with env(EDA_SWEEP_ML=64, EDA_SWEEP_K=2):
        with P.Handle.from_spec(spec, taps, precision=P.EDA_FP64) as h:
            h.eda_set_trajectory(xb, y)
            cols = torch.zeros(2, dtype=torch.int32, device=dev)
            V = torch.zeros(2, spec.n, dtype=torch.float64, device=dev)
            with pytest.raises(P.EdaError) as e:
                h.eda_hvp_noalloc(cols, V, torch.empty_like(V), True)
            assert e.value.code == P.EDA_ERR_INVALID and "multi-launch" in str(e.value)
