"""The allocation-free expectation entry point against the oracle and qaoa_expectation.

qaoa_expectation_noalloc serves callers that cannot allocate device memory (code
inside an allocator or pool callback, a teardown path, or a host that owns all
device memory): it takes its reduction scratch from a fixed array inside the
library instead of a caller workspace.  Three calls in a row share that array:
each result is checked against the FP64 oracle (or, at n = 28 where no CPU
statevector is practical, the p = 1 closed form) and against qaoa_expectation.
This file is collected last so that, if it fails, a run that stops at the first
failure has already run every other test.
"""
import ctypes as ct

import numpy as np
import pytest

import synth
from oracle import closed_form, qaoa

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


def test_noalloc_matches_oracle_three_calls():
    # call 1: complex128 QAOA state of a weighted graph, computed by the oracle and uploaded
    n1 = 14
    e, w, integer = synth.graph("gnp", n1, 3, weights="int", prob=0.4)
    C1 = qaoa.cut_values(n1, e, w)
    ref_state = qaoa.qaoa_state(n1, C1, *synth.angles(2, 1))
    cv1 = q.cost_vector(q.Graph(n1, e, w, integer), "i32")
    psi1 = torch.as_tensor(ref_state).cuda()
    lib1, got1 = _expect_both(psi1, cv1)
    scale = max(1.0, float(np.abs(w).sum()))
    E1 = qaoa.expectation(ref_state, C1)
    assert abs(got1[0] - E1) <= 1e-10 * scale and abs(got1[1] - qaoa.norm2(ref_state)) <= 1e-12
    assert abs(got1[0] - lib1[0]) <= 1e-12 * scale
    # call 2, right after: another size and dtype (complex64, float costs) reuses the scratch
    n2 = 20
    e2, w2, integer2 = synth.graph("reg3", n2, 5, weights="u01")
    C2 = qaoa.cut_values(n2, e2, w2, integer=False)
    cv2 = q.cost_vector(q.Graph(n2, e2, w2, integer2), "f64")
    psi2 = torch.as_tensor(synth.random_state(n2, 4)).to(torch.complex64).cuda()
    read2 = psi2.cpu().numpy().astype(np.complex128)  # the values the kernel reads
    lib2, got2 = _expect_both(psi2, cv2)
    E2 = qaoa.expectation(read2, C2)
    assert abs(got2[0] - E2) <= 1e-4 * max(1.0, abs(E2))
    assert abs(got2[1] - qaoa.norm2(read2)) <= 1e-4
    assert abs(got2[0] - lib2[0]) <= 1e-4 * max(1.0, abs(lib2[0]))
    del psi2, cv2
    # call 3: n = 28, complex128 (4.3 GB state, the largest reduction grid) after one QAOA
    # layer, whose <C> the per-edge closed form gives
    n3 = 28
    e3, w3, integer3 = synth.graph("reg3", n3, 2, weights="u01")
    cv3 = q.cost_vector(q.Graph(n3, e3, w3, integer3), "f64")
    gam, bet = synth.angles(1, 5)
    psi3 = q.new_state(n3, "c128")
    q.apply_layers(psi3, cv3, gam, bet)
    lib3, got3 = _expect_both(psi3, cv3)
    E3 = closed_form.expectation_p1(n3, e3, w3, gam[0], bet[0])
    scale3 = max(1.0, float(np.abs(w3).sum()))
    assert abs(got3[0] - E3) <= 1e-10 * scale3 and abs(got3[1] - 1.0) <= 1e-12
    assert abs(got3[0] - lib3[0]) <= 1e-12 * scale3
    del psi3, cv3
    torch.cuda.empty_cache()
