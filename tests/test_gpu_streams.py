"""Problems created and solved on a non-blocking side stream while the legacy
default stream is busy give the same results as on the default stream: every
device buffer is zero-filled and ready before the problem's own stream uses it."""
import numpy as np
import pytest

from paper_2110_15676_gb300 import workloads as W
from pairs import gpu_problem

pytestmark = pytest.mark.gpu


def _run(afc, wl, steps=3):
    g = gpu_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir)
    g.set_solution(wl.u0)
    dt = g.cfl_timestep(0.5)
    for _ in range(steps):
        g.step(afc.default_opts(scheme=afc.AFC_SSP3, dt=dt))
    u = g.get_solution()
    g.close()
    return dt, u


def test_side_stream_with_busy_default_stream():
    import torch
    from paper_2110_15676_gb300 import afc
    wl = W.random_transient(np.random.default_rng(60), "p1", (16, 16))
    dt_ref, u_ref = _run(afc, wl)
    a = torch.randn(4096, 4096, device="cuda")
    side = torch.cuda.Stream()
    for _ in range(3):
        for _ in range(20):           # keep the legacy default stream busy
            a = torch.tanh(a @ a * 1e-3)
        with torch.cuda.stream(side):
            dt, u = _run(afc, wl)
        assert dt == dt_ref
        assert np.array_equal(u, u_ref)
    torch.cuda.synchronize()
