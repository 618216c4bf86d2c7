"""The allocation-free output step (dgamp_ct_output_step_noalloc).

Callers that cannot allocate device memory while they run (a host that
reserves the whole GPU for its own memory pool, a latency-critical loop)
use this entry point: it needs no plan and keeps its scratch in a fixed
array inside the library.  This test calls it twice in a row through the C
ABI and checks both results against the plan-based dgamp_ct_output_step and
against the FP64 oracle's output step (Algorithm 1, Step 2), within the
tolerance the other output-step tests use (1e-5); it also checks that the
device's free memory does not change over repeated calls.  It lives in a
file of its own that pytest collects last, and it passes alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_04661_gb300 import build
    build.build()
    import paper_1609_04661_gb300 as dg
    dg.load()
    return dg


def _inputs(seed, nv, nd):
    rng = np.random.default_rng(seed)
    I0 = 1e5
    z_true = rng.uniform(0.0, 12.0, (nv, nd))
    y = rng.poisson(I0 * np.exp(-z_true)).astype(np.float32)
    z = (z_true + rng.normal(0, 0.5, (nv, nd))).astype(np.float32)
    s_prev = rng.normal(0, 1.0, (nv, nd)).astype(np.float32)
    return [torch.as_tensor(a).cuda() for a in (z, y, s_prev)], I0


def _oracle_step(z, y, s_prev, I0, tau_p):
    """The oracle's output step on the p the kernel forms in FP32 (p = z - tau_p s_prev)."""
    from oracle import output_step
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    zh, yh, sh = (t.cpu().numpy().reshape(-1) for t in (z, y, s_prev))
    p = f32(f32(zh) - f32(tau_p) * f32(sh))
    s_ref, tsi_ref, _, _ = output_step.output_step(p, yh.astype(np.float64), float(f32(tau_p)), I0)
    return s_ref, float(np.mean(tsi_ref))


def test_noalloc_output_step_matches_plan_path_twice(dg):
    from paper_1609_04661_gb300 import binding
    nv, nd = 37, 611                       # M = 22607: many blocks and a ragged tail
    with dg.Plan(16, nv, nd) as pl:
        for call, (seed, tau_p) in enumerate([(1, 0.05), (2, 2.0)]):
            (z, y, s_prev), I0 = _inputs(seed, nv, nd)
            s_ref, ts_ref = pl.output_step(z, y, s_prev, I0, tau_p)
            s = torch.empty_like(z)
            ts = torch.empty(1, dtype=torch.float64, device="cuda")
            binding.output_step_noalloc(z, y, s_prev, I0, tau_p, s, ts)
            torch.cuda.synchronize()
            a, b = s.cpu().numpy().astype(np.float64), s_ref.cpu().numpy().astype(np.float64)
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5, call
            assert float(ts.item()) == pytest.approx(float(ts_ref.item()), rel=1e-5), call
            so, tso = _oracle_step(z, y, s_prev, I0, tau_p)
            assert np.linalg.norm(a.reshape(-1) - so) / np.linalg.norm(so) < 1e-5, call
            assert float(ts.item()) == pytest.approx(tso, rel=1e-5), call


def test_noalloc_output_step_allocates_nothing(dg):
    """After a first call (which looks up the scratch address), further calls
    leave the device's free memory unchanged."""
    from paper_1609_04661_gb300 import binding
    (z, y, s_prev), I0 = _inputs(3, 29, 517)
    s = torch.empty_like(z)
    ts = torch.empty(1, dtype=torch.float64, device="cuda")
    binding.output_step_noalloc(z, y, s_prev, I0, 0.3, s, ts)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(8):
        binding.output_step_noalloc(z, y, s_prev if k % 2 else None, I0, 0.3 + 0.1 * k, s, ts)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_maximum(dg):
    from paper_1609_04661_gb300 import binding
    lib = binding.load()
    z = torch.zeros(8, device="cuda")
    ts = torch.empty(1, dtype=torch.float64, device="cuda")
    p = lambda t: binding.C.c_void_p(t.data_ptr())
    rc = lib.dgamp_ct_output_step_noalloc(p(z), p(z), None, (1 << 24) + 1, 1e5, 0.1, p(z), p(ts), None)
    assert rc == -1
    rc = lib.dgamp_ct_output_step_noalloc(p(z), p(z), None, 0, 1e5, 0.1, p(z), p(ts), None)
    assert rc == -1
