"""The entry point that allocates no device memory (afc_mc_limited_sum_noalloc).

Some callers cannot call cudaMalloc at the point where they need the limiter:
code that runs while a stream is being captured, or a runtime that reserves all
device memory at start-up.  This test calls the variant through the C ABI, twice
in a row with different states, and checks each result against the allocating
afc_mc_limited_sum, within the per-pass parity tolerance of the other tests.
It lives in a file of its own that is collected last."""
import numpy as np
import pytest

from paper_2110_15676_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PASS_TOL = 1e-13


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_15676_gb300 import afc
    return torch, afc


def _mc_problem(afc, elem, n):
    wl = W.stationary_inflow(elem, n)
    P = afc.Problem.structured(wl.elem, wl.n)
    P.set_coefficients(wl.eps, wl.b, wl.c, wl.f)
    P.set_dirichlet(wl.dir_mask, wl.u_dir)
    P.assemble(afc.AFC_FAMILY_MC, afc.AFC_FP64)
    return P


@pytest.mark.parametrize("elem,n", [("p1", 17), ("q1", 13)])
def test_noalloc_matches_allocating_entry_point_twice(cuda, elem, n):
    torch, afc = cuda
    P = _mc_problem(afc, elem, n)
    rng = np.random.default_rng(7)
    for call in range(2):                       # second call reuses the shared scratch
        u = rng.uniform(0, 1, P.N) if call == 0 else rng.normal(0.5, 0.3, P.N)
        ref = P.mc_limited_sum(u, afc.AFC_LIM_MC)["Fstar"]
        ud = torch.tensor(u, dtype=torch.float64, device="cuda")
        out = torch.full((P.N,), float("nan"), dtype=torch.float64, device="cuda")
        P.mc_limited_sum_noalloc(ud, out, afc.AFC_LIM_MC)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= PASS_TOL * scale, call
    for lim in (afc.AFC_LIM_GALERKIN, afc.AFC_LIM_NONE):
        ref = P.mc_limited_sum(u, lim)["Fstar"]
        P.mc_limited_sum_noalloc(ud, out, lim)
        torch.cuda.synchronize()
        assert np.abs(out.cpu().numpy() - ref).max() <= PASS_TOL * max(np.abs(ref).max(), 1e-300)


def test_noalloc_needs_the_mc_family(cuda):
    torch, afc = cuda
    wl = W.stationary_inflow("p1", 9)
    P = afc.Problem.structured(wl.elem, wl.n)
    P.set_coefficients(wl.eps, wl.b, wl.c, wl.f)
    P.set_dirichlet(wl.dir_mask, wl.u_dir)
    P.assemble(afc.AFC_FAMILY_FCT, afc.AFC_FP64)
    u = torch.zeros(P.N, dtype=torch.float64, device="cuda")
    out = torch.zeros(P.N, dtype=torch.float64, device="cuda")
    for lim in (afc.AFC_LIM_MC, afc.AFC_LIM_GALERKIN):
        with pytest.raises(afc.AfcError) as e:
            P.mc_limited_sum_noalloc(u, out, lim)
        assert e.value.status == afc.AFC_E_STATE
    P.mc_limited_sum_noalloc(u, out, afc.AFC_LIM_NONE)   # alpha = 0 needs no MC data
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0


def test_noalloc_rejects_sizes_beyond_its_scratch(cuda):
    torch, afc = cuda
    P = _mc_problem(afc, "p1", 65)              # 274,625 nodes > 262,144
    u = torch.zeros(P.N, dtype=torch.float64, device="cuda")
    out = torch.zeros(P.N, dtype=torch.float64, device="cuda")
    with pytest.raises(afc.AfcError) as e:
        P.mc_limited_sum_noalloc(u, out)
    assert e.value.status == afc.AFC_E_INVALID
    assert "262144" in str(e.value)
