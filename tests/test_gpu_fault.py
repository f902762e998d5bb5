"""Failure detection without a GPU fault.  Every wait of the fused kernels on a halo or
a copy is bounded; when the bound runs out the kernel sets the handle's device status
word and finishes, and the next synchronising call returns DD_TV_ETIMEOUT.  Here the
bound runs out on purpose (kind 0: one thread waits on an mbarrier phase that nothing
completes, no copy counted on it) or the word is written from the host (kind 1, a
corrupted word).  Afterwards the same handle solves again and matches a fresh handle
bit for bit: the context and the handle stay usable."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_00682_gb300 import _lib as L
    L.load()
    return L


def _solve(s, f, n):
    s.load(f, None)
    s.iterate(n)
    u = torch.empty_like(f)
    s.get_u(u)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("kind", [0, 1])
def test_timeout_path_reports_and_handle_recovers(kind):
    L = _lib()
    f = torch.from_numpy(synth.rof_image(256, 256, 12, 0.05, 0)[0]).cuda()
    s = L.Solver(L.make_params(256, 256, 2, 2))
    rc, msg, waited = s.fault_probe(kind)
    assert rc == L.ETIMEOUT, (rc, msg)
    assert "wait" in msg
    if kind == 0:
        print(f"bounded wait ran out after {waited:.1f} ms of device time")
        assert 0.0 < waited < 10_000.0
    else:
        assert waited == 0.0
    # the word was cleared: the handle solves, and exactly as a fresh one does
    u1 = _solve(s, f, 4)
    u2 = _solve(L.Solver(L.make_params(256, 256, 2, 2)), f, 4)
    assert np.array_equal(u1, u2)
    # a second probe fires again (nothing is latched)
    rc2, _, _ = s.fault_probe(1)
    assert rc2 == L.ETIMEOUT


def test_fault_probe_rejects_unknown_kind():
    L = _lib()
    s = L.Solver(L.make_params(64, 64, 1, 1))
    rc, msg, _ = s.fault_probe(7)
    assert rc == L.EINVAL and "kind" in msg
