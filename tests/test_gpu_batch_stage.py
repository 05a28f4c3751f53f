"""The persistent batched launch shapes (all passes of a stage, or of a step, in one
launch with grid barriers between the passes) against the same instances stepped
alone, bit for bit, on instances large enough that every block owns tiles of
several instances and reads, after each barrier, data other blocks wrote in the
launch's earlier passes.  Mixed precision, where the stage's float fluxes written
in the edge pass are read by the factor and correction passes of the same launch."""
import numpy as np
import pytest

from paper_2110_15676_gb300 import workloads as W
from pairs import gpu_problem

pytestmark = pytest.mark.gpu


def _gpu(wl, precision):
    g = gpu_problem(wl.elem, wl.n, wl.b, wl.eps, wl.c, wl.f, wl.dir_mask, wl.u_dir, precision=precision)
    g.set_solution(wl.u0)
    return g


@pytest.mark.parametrize("mode_name", ["PER_STAGE", "PER_STEP"])
def test_persistent_batched_mixed_equals_solo(mode_name):
    from paper_2110_15676_gb300 import afc
    mode = getattr(afc, "AFC_BATCH_" + mode_name)
    rng = np.random.default_rng(90)
    wls = [W.random_transient(rng, elem, (n, n)) for elem, n in (("q1", 81), ("p1", 64), ("q1", 33), ("p1", 20))]
    steps = 12
    solo = []
    dts = []
    for wl in wls:
        g = _gpu(wl, "mixed")
        dt = g.cfl_timestep(0.5)
        dts.append(dt)
        o = afc.default_opts(scheme=afc.AFC_SSP3, dt=dt, precision=afc.AFC_MIXED)
        for _ in range(steps):
            g.step(o)
        solo.append(g.get_solution())
        g.close()
    gs = [_gpu(wl, "mixed") for wl in wls]
    opts = afc.default_opts(scheme=afc.AFC_SSP3, precision=afc.AFC_MIXED)
    with afc.Batch(gs) as b:
        for blk in (512, 256):
            for g, wl in zip(gs, wls):
                g.set_solution(wl.u0)
            b.set_tuning(mode, blk)
            b.step(opts, dt=dts, nsteps=steps)
            for q, g in enumerate(gs):
                u = g.get_solution()
                assert np.array_equal(u, solo[q]), (mode_name, blk, q, float(np.abs(u - solo[q]).max()))
    for g in gs:
        g.close()


def test_batched_mixed_instances_on_their_own_streams_equal_solo():
    """Instances created on their own streams, batched on the first one's stream while
    other work keeps the GPU busy on a third stream: the single-precision copies that
    the first mixed batched step makes are enqueued on each instance's stream, and the
    batch's stream must not read them before they are done."""
    import torch
    from paper_2110_15676_gb300 import afc
    rng = np.random.default_rng(91)
    wls = [W.random_transient(rng, elem, (n, n)) for elem, n in (("q1", 41), ("q1", 81), ("p1", 64))]
    steps = 4
    solo, dts = [], []
    for wl in wls:
        g = _gpu(wl, "mixed")
        dt = g.cfl_timestep(0.5)
        dts.append(dt)
        o = afc.default_opts(scheme=afc.AFC_SSP3, dt=dt, precision=afc.AFC_MIXED)
        for _ in range(steps):
            g.step(o)
        solo.append(g.get_solution())
        g.close()
    opts = afc.default_opts(scheme=afc.AFC_SSP3, precision=afc.AFC_MIXED)
    busy = torch.cuda.Stream()
    a = torch.randn(4096, 4096, device="cuda")
    for trial in range(3):
        streams = [torch.cuda.Stream() for _ in wls]
        gs = []
        for wl, st in zip(wls, streams):
            with torch.cuda.stream(st):
                gs.append(_gpu(wl, "mixed"))
        with torch.cuda.stream(busy):
            for _ in range(40):
                a = torch.tanh(a @ a * 1e-3)
        with afc.Batch(gs) as b:
            b.set_tuning(afc.AFC_BATCH_PER_STAGE, 256)
            b.step(opts, dt=dts, nsteps=steps)
            for q, g in enumerate(gs):
                u = g.get_solution()
                assert np.array_equal(u, solo[q]), (trial, q, float(np.abs(u - solo[q]).max()))
        for g in gs:
            g.close()
    torch.cuda.synchronize()
