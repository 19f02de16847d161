"""Invariants of the multigrid kernels, checked on the GPU through the C ABI.

* The fused schedule (wavefront kernels that pipeline all nu red-black half-sweeps, the
  residual and the restriction in one pass per level, plus the one-CTA coarse tail) performs
  exactly the arithmetic of the reference schedule (one kernel per half-sweep, restriction
  and prolongation): outputs and statistics must be bit-identical.
* Results do not depend on how the slices are batched (ragged batch vs one call per slice).
"""
import pytest
import torch

from paper_1506_02079_gb300 import api
from paper_1506_02079_gb300.synthetic import make_stack, make_ragged_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib()
    return torch.device("cuda", 0)


def solve(s, o, alpha, **kw):
    return api.emfuse_screened_poisson(s, o, alpha, api.default_opts(**kw), return_stats=True,
                                       allow_noconv=True)


@pytest.mark.parametrize("shape", [(4, 256, 256), (3, 300, 517), (2, 129, 1000), (5, 65, 70), (1, 1, 1)])
@pytest.mark.parametrize("nu", [(1, 1), (2, 2), (3, 3), (2, 1), (1, 3), (3, 4), (2, 4), (4, 2)])
@pytest.mark.parametrize("precision", [api.PREC_FP32, api.PREC_MIXED, api.PREC_FP64])
def test_fused_equals_reference_schedule(dev, shape, nu, precision):
    I0 = make_stack(*shape, seed=21).to(dev)
    s = api.emfuse_smooth_z(I0, 1.0, 3.0)
    kw = dict(nu_pre=nu[0], nu_post=nu[1], precision=precision, max_vcycles=3, tol=0.0)
    fa, sa = solve(s, I0, 1e-3, fused=1, **kw)
    fb, sb = solve(s, I0, 1e-3, fused=0, **kw)
    assert torch.equal(fa, fb)
    # residual norms are summed with atomics: equal up to the summation order
    for x, y in zip(sa, sb):
        assert x["rel_residual"] == pytest.approx(y["rel_residual"], rel=1e-12, abs=1e-300)


def test_fused_equals_reference_ragged(dev):
    sides = [(1, 1), (2, 3), (64, 64), (65, 64), (130, 257), (300, 37), (513, 200), (1024, 97)]
    s, o, ny, nx, offs = make_ragged_batch(len(sides), seed=5, sides=sides)
    s, o = s.to(dev), o.to(dev)
    kw = dict(max_vcycles=4, tol=0.0)
    fa, sa = api.emfuse_screened_poisson(s, o, 1e-2, api.default_opts(fused=1, **kw), nx=nx, ny=ny,
                                         offsets=offs, return_stats=True, allow_noconv=True)
    fb, sb = api.emfuse_screened_poisson(s, o, 1e-2, api.default_opts(fused=0, **kw), nx=nx, ny=ny,
                                         offsets=offs, return_stats=True, allow_noconv=True)
    assert torch.equal(fa, fb)


def test_batching_does_not_change_results(dev):
    sides = [(70, 90), (256, 256), (33, 400)]
    s, o, ny, nx, offs = make_ragged_batch(len(sides), seed=6, sides=sides)
    s, o = s.to(dev), o.to(dev)
    opts = api.default_opts(max_vcycles=5, tol=0.0)
    fa = api.emfuse_screened_poisson(s, o, 1e-3, opts, nx=nx, ny=ny, offsets=offs, allow_noconv=True)
    for j in range(len(sides)):
        a, h, w = int(offs[j]), int(ny[j]), int(nx[j])
        fj = api.emfuse_screened_poisson(s[a:a + h * w].view(h, w), o[a:a + h * w].view(h, w), 1e-3,
                                         opts, allow_noconv=True)
        assert torch.equal(fj.reshape(-1), fa[a:a + h * w])


def test_vcycle_contraction(dev):
    """Per-V-cycle residual reduction on the EM-like data at the paper's alpha = 0.001: the
    solver table of Sec. 4 reports decays of 0.23 / 0.11 / 0.04 per V-cycle for its FEM
    discretisations; this FV multigrid must do at least as well as the best of them."""
    I0 = make_stack(4, 512, 512, seed=1).to(dev)
    s = api.emfuse_smooth_z(I0, 1.0, 3.0)
    res = []
    for v in range(0, 5):
        _, st = solve(s, I0, 1e-3, max_vcycles=v, tol=0.0, precision=api.PREC_FP64)
        res.append(max(x["rel_residual"] for x in st))
    rates = [res[i + 1] / res[i] for i in range(len(res) - 1)]
    assert max(rates) < 0.1, rates


def test_integer_pipe_conversions_match_hardware(dev):
    """The residual kernels widen and round between FP32 and FP64 with integer operations;
    every binary32 pattern and 7 x 2^32 binary64 patterns must match the hardware bit for bit."""
    assert api.emfuse_selftest_fpconv() == (0, 0)


def test_device_code_is_sm103a_and_fp64_probe_runs(dev):
    """The loaded device code is sm_103a (binary version 103, a runtime query instead of any
    look into the binary); the FP64 rate probe returns a plausible GB300 rate (nominal 1.25
    TFLOP/s at the maximum clock; well above 0.1 and below 3 at any clock)."""
    assert api.emfuse_kernel_binary_version() == 103
    r = api.emfuse_probe_fp64_fma_rate(dev)
    assert 0.1 < r < 3.0, r


def test_slices_met_at_initial_iterate_return_o(dev):
    """A slice with s = o has r = 0 at f = o and is never iterated; its output must still be
    written (f = o) while the other slices of the batch iterate, in every precision."""
    I0 = make_stack(3, 96, 80, seed=4).to(dev)
    s = api.emfuse_smooth_z(I0, 1.0, 3.0)
    s[1] = I0[1]
    for prec in (api.PREC_FP32, api.PREC_MIXED, api.PREC_FP64):
        f, st = solve(s, I0, 1e-2, precision=prec)
        assert st[1]["vcycles"] == 0 and st[0]["vcycles"] > 0
        assert torch.equal(f[1], I0[1])
        f0, _ = solve(s, I0, 1e-2, precision=prec, max_vcycles=0)
        assert torch.equal(f0, I0)


@pytest.mark.parametrize("precision", [api.PREC_FP32, api.PREC_MIXED])
def test_graph_replay_and_tile_rows_are_bit_identical(dev, precision):
    """Replaying the V-cycle as a CUDA graph, and any rows-per-work-item on the finest level,
    give exactly the directly launched result."""
    s, o, ny, nx, offs = make_ragged_batch(9, seed=6, side_lo=40, side_hi=700)
    s, o = s.to(dev), o.to(dev)
    def run(**kw):
        return api.emfuse_screened_poisson(s, o, 1e-3, api.default_opts(precision=precision, **kw), nx=nx, ny=ny,
                                           offsets=offs, return_stats=True)
    f0, st0 = run(no_graphs=1)
    for kw in (dict(), dict(tile_rows=8), dict(tile_rows=32), dict(tile_rows=256), dict(no_graphs=1, tile_rows=64)):
        f1, st1 = run(**kw)
        assert torch.equal(f1, f0), kw
        assert [a["vcycles"] for a in st1] == [a["vcycles"] for a in st0]
    # a graph captured for one alpha is not replayed for another
    g1 = api.emfuse_screened_poisson(s, o, 0.1, api.default_opts(precision=precision), nx=nx, ny=ny, offsets=offs)
    g2 = api.emfuse_screened_poisson(s, o, 0.1, api.default_opts(precision=precision, no_graphs=1), nx=nx, ny=ny,
                                     offsets=offs)
    assert torch.equal(g1, g2)


@pytest.mark.parametrize("precision", [api.PREC_MIXED, api.PREC_FP64])
def test_async_solve_returns_before_the_gpu_and_matches_the_blocking_call(dev, precision):
    """opts.async_solve = 1: the whole solve (its outer loop a WHILE node of one CUDA graph) is
    queued and the call returns while the GPU still works; after a stream synchronisation the
    output is bit-identical to the blocking call's and the stats equal its stats.  A slice that
    cannot reach tol is reported through stats.converged = 0 (no status code)."""
    I0 = make_stack(16, 1024, 1024, seed=9).to(dev)
    s = api.emfuse_smooth_z(I0, 1.0, 3.0)
    ref, st_ref = api.emfuse_screened_poisson(s, I0, 1e-3, api.default_opts(precision=precision), return_stats=True)
    stream = torch.cuda.current_stream(dev)
    opts = api.default_opts(precision=precision, async_solve=1)
    api.emfuse_screened_poisson(s, I0, 1e-3, opts)  # the first call of a geometry builds its plan and graph
    torch.cuda.synchronize(dev)
    out = torch.full_like(I0, float("nan"))
    f, pending = api.emfuse_screened_poisson(s, I0, 1e-3, opts, out=out, return_stats=True)
    ev = torch.cuda.Event()
    ev.record(stream)
    still_running = not ev.query()
    st = pending.result()
    assert still_running
    assert torch.equal(f, ref)
    assert st == st_ref
    # non-convergence: no status code, converged = 0 in the stats
    few = api.default_opts(precision=precision, async_solve=1, max_vcycles=1)
    _, pend = api.emfuse_screened_poisson(s, I0, 1e-3, few, return_stats=True)
    st1 = pend.result()
    assert all(a["vcycles"] == 1 and not a["converged"] for a in st1)


def test_autotune_picks_the_fastest_candidate(dev):
    s, o, ny, nx, offs = make_ragged_batch(10, seed=2, side_lo=64, side_hi=900)
    s, o = s.to(dev), o.to(dev)
    f, st = api.emfuse_screened_poisson(s, o, 1e-3, api.default_opts(autotune=1), nx=nx, ny=ny, offsets=offs,
                                        return_stats=True)
    table = api.emfuse_autotune_result()
    assert len(table) == 20
    # one to four sweeps per leg, each sweep count with two tile heights (rows per work item)
    pairs = {(e["nu_pre"], e["nu_post"]) for e in table}
    assert pairs >= {(1, 1), (2, 2), (3, 3), (3, 4), (2, 3), (3, 2), (4, 4)}
    for nu in pairs:
        assert len({e["tile_rows"] for e in table if (e["nu_pre"], e["nu_post"]) == nu}) >= 2, nu
    best = table[0]
    assert best["ms"] == min(e["ms"] for e in table if e["ms"] >= 0)
    ref = api.emfuse_screened_poisson(s, o, 1e-3, api.default_opts(nu_pre=best["nu_pre"], nu_post=best["nu_post"],
                                                                    tile_rows=best["tile_rows"]),
                                      nx=nx, ny=ny, offsets=offs)
    assert torch.equal(f, ref)
    assert all(a["converged"] for a in st)


def test_bounded_wait_runs_out_and_context_stays_usable(dev):
    """A device wait on a barrier that nothing completes gives up after its poll limit: the
    call reports EMFUSE_ETIMEOUT (5) and clears the device error word, and the context then
    runs a solve and the self-test again as before (no fault, no hang: the wait is bounded)."""
    L = api.lib()
    st = torch.cuda.current_stream(dev).cuda_stream
    assert L.emfuse_selftest_wait_timeout(1000, st) == 5
    assert b"ran out" in L.emfuse_last_error()
    I0 = make_stack(2, 64, 48, seed=21).to(dev)
    f, stats = api.emfuse_screened_poisson(I0, I0.flip(0).contiguous(), 0.01, return_stats=True)
    assert all(s["converged"] for s in stats) and bool(torch.isfinite(f).all())
    assert L.emfuse_selftest_wait_timeout(1, st) == 5
