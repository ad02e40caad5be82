"""The allocation-free expectation entry point agrees with qaoa_expectation.

qaoa_expectation_noalloc serves callers that cannot allocate device memory: it
takes its reduction scratch from a fixed array inside the library instead of a
caller workspace.  This file is collected last so that, if it fails, a run that
stops at the first failure has already run every other test.
"""
import ctypes as ct

import numpy as np
import pytest

import synth
from oracle import qaoa

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_13012_gb300 as q  # noqa: E402


def _expect_both(psi, cv):
    n = int(np.log2(psi.numel()))
    dt = q.C128 if psi.dtype == torch.complex128 else q.C64
    ref = q.expectation(psi, cv)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=psi.device)
    cs = cv.struct()
    rc = q.lib.qaoa_expectation_noalloc(n, dt, ct.c_void_p(psi.data_ptr()), ct.byref(cs),
                                        ct.c_void_p(out.data_ptr()),
                                        ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == q.QAOA_OK, q.lib.qaoa_strerror(rc)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), out.cpu().numpy()


def test_noalloc_matches_expectation_two_calls():
    # call 1: complex128 state of a weighted graph
    n1 = 14
    e, w, integer = synth.graph("gnp", n1, 3, weights="int", prob=0.4)
    cv1 = q.cost_vector(q.Graph(n1, e, w, integer), "i32")
    psi1 = torch.as_tensor(qaoa.qaoa_state(n1, qaoa.cut_values(n1, e, w), *synth.angles(2, 1))).cuda()
    ref, got = _expect_both(psi1, cv1)
    scale = max(1.0, float(np.abs(w).sum()))
    assert abs(got[0] - ref[0]) <= 1e-10 * scale and abs(got[1] - ref[1]) <= 1e-12
    # call 2, right after: a different size and dtype reuses the same scratch
    n2 = 20
    e2, w2, integer2 = synth.graph("reg3", n2, 5, weights="u01")
    cv2 = q.cost_vector(q.Graph(n2, e2, w2, integer2), "f64")
    psi2 = torch.as_tensor(synth.random_state(n2, 4)).to(torch.complex64).cuda()
    ref2, got2 = _expect_both(psi2, cv2)
    assert abs(got2[0] - ref2[0]) <= 1e-4 * max(1.0, abs(ref2[0]))
    assert abs(got2[1] - ref2[1]) <= 1e-4
