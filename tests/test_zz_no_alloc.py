"""The allocation-free energy entry point (dd_tv_energy_noalloc).

Some callers cannot allocate device memory when they need an energy value (their
device memory is held by another framework's pool, or cudaMalloc's implicit
synchronisation is not allowed in their loop).  dd_tv_energy_noalloc runs the same
reduction with scratch in a fixed array inside the library.  This file is collected
last so that a failure here never hides the other tests; it passes alone in a fresh
process and after them.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _energy_noalloc(lib, u, f, mask, fid, alpha, c1, c2, stream):
    J = ctypes.c_double()
    rc = lib.dd_tv_energy_noalloc(u.data_ptr(), f.data_ptr(), None if mask is None else mask.data_ptr(),
                                  u.shape[0], u.shape[1], fid, alpha, c1, c2, ctypes.c_void_p(stream),
                                  ctypes.byref(J))
    return rc, J.value


def test_noalloc_energy_matches_handle_energy_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_00682_gb300 import _lib as L
    lib = L.load()
    stream = torch.cuda.current_stream().cuda_stream
    tv_f, tv_mask, _ = synth.tvl1_inpaint_image(256, 192, 12, 0.1, 0.2, 22)
    cases = [
        # odd width: the per-pixel reduction kernel
        (synth.rof_image(300, 517, 20, 0.05, 21)[0], None, L.L2, 8.0, 0.0, 0.0),
        # width a multiple of 4 with a mask, then without: the two row-kernel instances
        (tv_f, tv_mask, L.L1, 1.5, 0.0, 0.0),
        (synth.rof_image(200, 320, 15, 0.05, 23)[0], None, L.SEG, 20.0, 0.2, 0.8),
    ]
    for f, mask, fid, alpha, c1, c2 in cases:   # calls in a row, different images
        H, W = f.shape
        rng = np.random.default_rng(H)
        u = torch.from_numpy((f + 0.02 * rng.standard_normal(f.shape)).astype(np.float32)).cuda()
        fd = torch.from_numpy(f).cuda()
        md = None if mask is None else torch.from_numpy(mask).cuda()
        rc, J = _energy_noalloc(lib, u, fd, md, fid, alpha, c1, c2, stream)
        assert rc == L.OK
        s = L.Solver(L.make_params(H, W, fidelity=fid, alpha=alpha, c1=c1, c2=c2, path="fulldim"))
        J_ref = s.energy(u, fd, md)
        s.close()
        assert abs(J - J_ref) <= 1e-6 * abs(J_ref), (J, J_ref)
        # and against the FP64 oracle's energy of the same float32 arrays
        fidname = {L.L2: "l2", L.L1: "l1", L.SEG: "seg"}[fid]
        pr = oracle.Problem(H, W, fidelity=fidname, alpha=alpha, c1=c1, c2=c2)
        Jo = oracle.energy(pr, u.cpu().numpy().astype(np.float64), f.astype(np.float64), mask)
        assert abs(J - Jo) <= 1e-5 * abs(Jo), (J, Jo)


def test_noalloc_energy_rejects_bad_sizes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_00682_gb300 import _lib as L
    lib = L.load()
    u = torch.zeros(4, 4, device="cuda")
    J = ctypes.c_double()
    assert lib.dd_tv_energy_noalloc(u.data_ptr(), u.data_ptr(), None, 0, 4, L.L2, 1.0, 0.0, 0.0, None,
                                    ctypes.byref(J)) == L.EINVAL
    assert lib.dd_tv_energy_noalloc(u.data_ptr(), u.data_ptr(), None, 65536, 65536, L.L2, 1.0, 0.0, 0.0, None,
                                    ctypes.byref(J)) == L.EINVAL
