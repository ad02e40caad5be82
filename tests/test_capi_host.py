"""Host-side checks of the C ABI: the library loads, exports every declared symbol,
and rejects bad input before any GPU work (no GPU needed)."""
import ctypes as ct
import re
from pathlib import Path

import numpy as np
import pytest

import paper_2407_13012_gb300 as q

HEADERS = sorted((Path(__file__).resolve().parent.parent / "include").glob("*.h"))


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names |= set(re.findall(r"\b(qaoa_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 16
    lib = ct.CDLL(str(q._LIB_PATH))
    for name in names:
        assert hasattr(lib, name), name
    assert set(q.EXPORTS) <= set(names)


def test_version_and_strerror():
    assert q.version() >= 100
    for s in range(6):
        assert q.lib.qaoa_strerror(s)
    assert q.lib.qaoa_strerror(99) == b"unknown status"


def check(n, edges, weights=None, integer=True):
    g = q.Graph(n, np.asarray(edges).reshape(-1, 2), weights, integer)
    st = g.as_struct()
    lo, hi = ct.c_int64(), ct.c_int64()
    return q.lib.qaoa_graph_check(ct.byref(st), ct.byref(lo), ct.byref(hi)), lo.value, hi.value


def test_graph_check_accepts_and_bounds():
    rc, lo, hi = check(4, [[0, 1], [1, 2], [2, 3]], [2.0, -3.0, 5.0])
    assert rc == 0 and lo == -3 and hi == 7
    rc, lo, hi = check(4, np.zeros((0, 2)))
    assert rc == 0 and lo == 0 and hi == 0


@pytest.mark.parametrize("n,edges,weights,integer", [
    (4, [[0, 0]], None, True),             # loop
    (4, [[0, 4]], None, True),             # vertex out of range
    (4, [[0, -1]], None, True),            # negative vertex
    (4, [[0, 1], [1, 0]], None, True),     # repeated edge, other orientation
    (4, [[2, 3], [0, 1], [2, 3]], None, True),  # repeated edge, same orientation
    (32, [[31, 0], [5, 31], [0, 31]], None, True),  # repeated edge on the highest vertex
    (4, [[0, 1]], [1.5], True),            # non-integral weight under INT
    (4, [[0, 1]], [float("nan")], False),  # non-finite weight
    (4, [[0, 1]], [float("inf")], False),
    (0, np.zeros((0, 2)), None, True),     # n out of range
    (33, np.zeros((0, 2)), None, True),
    (3, [[0, 1]], [2.0 ** 31], True),      # integer sum overflows int32
])
def test_graph_check_rejects(n, edges, weights, integer):
    rc, _, _ = check(n, edges, weights, integer)
    assert rc == q.QAOA_ERR_INVALID_ARG


def test_graph_check_accepts_the_highest_vertices():
    rc, lo, hi = check(32, [[31, 0], [30, 31], [0, 1], [1, 30]], [1.0, 2.0, 3.0, 4.0])
    assert rc == 0 and lo == 0 and hi == 10


def test_graph_descriptor_follows_replaced_arrays():
    """The binding builds a graph's C descriptor once; replacing the edges or the weights gives
    a new one that points at the new arrays."""
    g = q.Graph(4, np.array([[0, 1], [1, 2]]), np.array([1.0, 2.0]))
    d1 = g.as_struct()
    assert g.as_struct() is d1 and d1.m == 2
    g.edges = np.ascontiguousarray(np.array([[0, 1], [1, 2], [2, 3]], dtype=np.int32))
    d2 = g.as_struct()
    assert d2 is not d1 and d2.m == 3 and d2.uv[4] == 2 and d2.uv[5] == 3
    g.weights = np.array([1.0, 2.0, 5.0])
    d3 = g.as_struct()
    assert d3 is not d2 and d3.w[2] == 5.0
    lo_hi = g.check()
    assert lo_hi == (0, 8)


def test_workspace_sizes():
    assert q.workspace_size(20, q.C128, q.OP_COST) == 0
    a = q.workspace_size(20, q.C128, q.OP_LAYERS, 4, 0, 0)
    b = q.workspace_size(20, q.C128, q.OP_LAYERS, 4, 0, 100)
    assert b > a > 0 and b % 256 == 0
    assert q.workspace_size(30, q.C64, q.OP_SAMPLE, 0, 10**6) > 8 * (1 << 20)
    g2 = q.workspace_size(24, q.C128, q.OP_GRADIENT, 10, 0, 0)
    assert g2 > q.workspace_size(24, q.C128, q.OP_GRADIENT, 1, 0, 0)
    out = ct.c_size_t()
    assert q.lib.qaoa_workspace_size(40, 0, 1, 1, 0, 0, ct.byref(out)) == q.QAOA_ERR_INVALID_ARG
    assert q.lib.qaoa_workspace_size(10, 0, 1, 65, 0, 0, ct.byref(out)) == q.QAOA_ERR_INVALID_ARG
    assert q.lib.qaoa_workspace_size(10, 7, 1, 1, 0, 0, ct.byref(out)) == q.QAOA_ERR_INVALID_ARG


def test_calls_reject_bad_arguments_before_launch():
    # argument errors are reported on the host; null pointers never reach a kernel
    dp = ct.POINTER(ct.c_double)
    g = np.array([0.1]), np.array([0.2])
    gp, bp = g[0].ctypes.data_as(dp), g[1].ctypes.data_as(dp)
    cost = q.CostT(0, q.COST_I32, 0, 1)
    assert q.lib.qaoa_apply_layers(10, q.C128, None, ct.byref(cost), gp, bp, 1, 1, None, None, 0, None) \
        == q.QAOA_ERR_INVALID_ARG
    cost = q.CostT(1 << 20, q.COST_I32, 0, 1)  # non-null but never dereferenced on these paths
    assert q.lib.qaoa_apply_layers(10, 5, ct.c_void_p(1 << 20), ct.byref(cost), gp, bp, 1, 1, None, None, 0,
                                   None) == q.QAOA_ERR_INVALID_ARG
    nan = np.array([np.nan])
    assert q.lib.qaoa_apply_layers(10, q.C128, ct.c_void_p(1 << 20), ct.byref(cost), nan.ctypes.data_as(dp), bp, 1,
                                   1, None, None, 0, None) == q.QAOA_ERR_INVALID_ARG
    assert q.lib.qaoa_apply_layers(10, q.C128, ct.c_void_p(1 << 20), ct.byref(cost), gp, bp, 65, 1, None, None, 0,
                                   None) == q.QAOA_ERR_INVALID_ARG
    # workspace too small
    assert q.lib.qaoa_apply_layers(10, q.C128, ct.c_void_p(1 << 20), ct.byref(cost), gp, bp, 1, 1, None,
                                   ct.c_void_p(1 << 21), 16, None) == q.QAOA_ERR_WORKSPACE
    assert q.lib.qaoa_gradient(10, q.C128, ct.c_void_p(1 << 20), ct.c_void_p(1 << 20), ct.byref(cost), gp, bp, 1,
                               ct.c_void_p(1 << 22), ct.c_void_p(1 << 21), 1 << 30, None) == q.QAOA_ERR_INVALID_ARG
    assert q.lib.qaoa_sample(10, q.C128, ct.c_void_p(1 << 20), ct.byref(cost), -1, 0, None, None, None, 0, None) \
        == q.QAOA_ERR_INVALID_ARG


# ---------------------------------------------------------------- batched gradients

def _batch_ws(graphs, p=3, dtype=q.C128, tiles=None):
    structs = (q.GraphT * max(len(graphs), 1))(*[g.as_struct() for g in graphs])
    tp = None
    if tiles is not None:
        tiles = np.ascontiguousarray(np.asarray(tiles, dtype=np.int32))
        tp = ct.c_void_p(tiles.ctypes.data)
    out = ct.c_size_t()
    rc = q.lib.qaoa_batch_workspace_size(dtype, p, len(graphs), structs, tp, ct.byref(out))
    return rc, out.value


def _ring(n, w=None, integer=True):
    e = np.array([[u, (u + 1) % n] for u in range(n)])
    return q.Graph(n, e, np.asarray(w if w is not None else np.ones(n)), integer)


def test_batch_workspace_sizes():
    rc, b1 = _batch_ws([_ring(10)])
    assert rc == 0 and b1 > 0
    rc, b2 = _batch_ws([_ring(10), _ring(16)])
    assert rc == 0
    # states, lambda and costs of the n = 16 graph: (16 + 16 + 4) bytes x 2^16 at least
    assert b2 - b1 >= 36 * 2 ** 16
    rc, b3 = _batch_ws([_ring(10), _ring(16)], dtype=q.C64)
    assert rc == 0 and b3 < b2
    rc, b0 = _batch_ws([])
    assert rc == 0
    # a float-weight graph makes every cost float64: 4 more bytes per amplitude
    rc, bf = _batch_ws([_ring(10), _ring(16, np.full(16, 0.5), integer=False)])
    assert rc == 0 and bf - b2 >= 4 * 2 ** 16


@pytest.mark.parametrize("case", ["too_big", "p_zero", "p_large", "bad_tile", "bad_graph"])
def test_batch_rejections(case):
    tiles = None
    graphs, p, want = [_ring(8)], 3, q.QAOA_ERR_INVALID_ARG
    if case == "too_big":
        graphs, want = [_ring(q.BATCH_MAX_N + 1)], q.QAOA_ERR_UNSUPPORTED
    elif case == "p_zero":
        p = 0
    elif case == "p_large":
        p = q.BATCH_MAX_P + 1
    elif case == "bad_tile":
        tiles = np.full(q.MAX_N + 1, 2)
    elif case == "bad_graph":
        graphs = [q.Graph(4, np.array([[0, 0]]), None, True)]
    rc, _ = _batch_ws(graphs, p=p, tiles=tiles)
    assert rc == want


def test_batch_gradient_checks_arguments_before_gpu_work():
    g = _ring(8)
    structs = (q.GraphT * 1)(g.as_struct())
    ang = np.zeros(6)
    dp = ang.ctypes.data_as(ct.POINTER(ct.c_double))
    # missing angles, then a workspace that is too small: both refused on the host
    assert q.lib.qaoa_batch_gradient(q.C128, 1, structs, None, 3, None, None, None, 0, None) == q.QAOA_ERR_INVALID_ARG
    assert q.lib.qaoa_batch_gradient(q.C128, 1, structs, dp, 3, None, None, None, 0, None) == q.QAOA_ERR_WORKSPACE
    ang[2] = float("nan")
    assert q.lib.qaoa_batch_gradient(q.C128, 1, structs, dp, 3, None, None, None, 0, None) == q.QAOA_ERR_INVALID_ARG
    size = ct.c_size_t()
    assert q.lib.qaoa_batch_autotune_workspace_size(q.C128, 3, 12, 4, ct.byref(size)) == 0 and size.value > 0
    assert q.lib.qaoa_batch_autotune_workspace_size(q.C128, 3, q.BATCH_MAX_N + 1, 4, ct.byref(size)) != 0


# ---------------------------------------------------------------- general PUBO cost

@pytest.mark.parametrize("case", ["var_outside", "nan", "non_integral", "i32_float", "no_masks", "n_zero"])
def test_pubo_rejections(case):
    n, masks, w, kind, cdt = 4, [0b0011, 0b1000], [1.0, -2.0], q.WEIGHT_INT, q.COST_I32
    if case == "var_outside":
        masks = [0b10000]
    elif case == "nan":
        w, kind, cdt = [float("nan"), 1.0], q.WEIGHT_F64, q.COST_F64
    elif case == "non_integral":
        w = [0.5, 1.0]
    elif case == "i32_float":
        kind = q.WEIGHT_F64
    elif case == "n_zero":
        n = 0
    m = np.ascontiguousarray(np.asarray(masks, dtype=np.uint32))
    wa = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    mp = None if case == "no_masks" else ct.c_void_p(m.ctypes.data)
    desc = q.CostT()
    # a placeholder device pointer: every case is refused on the host before any launch
    rc = q.lib.qaoa_cost_vector_pubo(n, len(m), mp, wa.ctypes.data_as(ct.POINTER(ct.c_double)), kind,
                                     ct.c_void_p(256), cdt, ct.byref(desc), None)
    assert rc == q.QAOA_ERR_INVALID_ARG


def test_optimizer_state_sizes_and_resume_checks():
    size = ct.c_size_t()
    assert q.lib.qaoa_optimizer_state_size(q.OPTIMIZER_ADAM, 4, ct.byref(size)) == 0
    assert size.value == (4 * 4 + 1) * 8
    assert q.lib.qaoa_optimizer_state_size(q.OPTIMIZER_LBFGS, 4, ct.byref(size)) == 0
    m, np2 = q.LBFGS_MAX_M, 8
    assert size.value == (16 + 3 * np2 + 2 * m * np2 + m) * 8
    assert q.lib.qaoa_optimizer_state_size(7, 4, ct.byref(size)) == q.QAOA_ERR_INVALID_ARG
    assert q.lib.qaoa_optimizer_state_size(q.OPTIMIZER_ADAM, 0, ct.byref(size)) == q.QAOA_ERR_INVALID_ARG
    # resume without a state buffer is refused on the host
    cost = q.CostT(256, q.COST_F64, 1, 0)
    ang = ct.c_void_p(512)
    assert q.lib.qaoa_optimize_adam(8, q.C128, None, None, ct.byref(cost), ang, 2, 5, 0.01, 0.9, 0.999, 1e-8,
                                    None, None, 1, None, 0, None) == q.QAOA_ERR_INVALID_ARG
    assert q.lib.qaoa_optimize_lbfgs(8, q.C128, None, None, ct.byref(cost), ang, 2, 5, 4, 1e-6, None, None,
                                     None, 1, None, 0, None) == q.QAOA_ERR_INVALID_ARG


def test_xy_dim_and_workspace_sizes():
    from math import comb
    d = ct.c_int64()
    for n, k in [(1, 0), (1, 1), (10, 3), (32, 16), (36, 18), (40, 20)]:
        assert q.lib.qaoa_xy_dim(n, k, ct.byref(d)) == 0 and d.value == comb(n, k)
        assert q.xy_dim(n, k) == comb(n, k)
    for n, k in [(0, 0), (41, 1), (5, -1), (5, 6)]:
        assert q.lib.qaoa_xy_dim(n, k, ct.byref(d)) == q.QAOA_ERR_INVALID_ARG
    b0, b1, b2 = ct.c_size_t(), ct.c_size_t(), ct.c_size_t()
    assert q.lib.qaoa_xy_workspace_size(20, 10, q.C128, 0, 0, ct.byref(b0)) == 0
    assert q.lib.qaoa_xy_workspace_size(20, 10, q.C128, 4, 100, ct.byref(b1)) == 0
    assert q.lib.qaoa_xy_workspace_size(20, 10, q.C64, 4, 100, ct.byref(b2)) == 0
    assert b0.value % 256 == 0 and b1.value >= b0.value + 4 * 100 * 16 and b2.value >= b0.value + 4 * 100 * 8
    assert q.lib.qaoa_xy_workspace_size(20, 10, 7, 0, 0, ct.byref(b0)) == q.QAOA_ERR_INVALID_ARG
    assert q.lib.qaoa_xy_workspace_size(20, 10, q.C128, q.MAX_P + 1, 0, ct.byref(b0)) == q.QAOA_ERR_INVALID_ARG


def test_xy_calls_reject_bad_arguments_before_launch():
    fake = ct.c_void_p(1 << 20)  # never dereferenced: every call below fails its checks first
    g = q.Graph(4, np.array([[0, 1], [1, 2]]), np.array([1.5, 2.0]), integer=False).as_struct()
    desc = q.CostT()
    # float weights with int32 costs, k out of range, no output
    assert q.lib.qaoa_xy_cost_vector(ct.byref(g), 2, fake, q.COST_I32, ct.byref(desc), None) == q.QAOA_ERR_INVALID_ARG
    assert q.lib.qaoa_xy_cost_vector(ct.byref(g), 5, fake, q.COST_F64, ct.byref(desc), None) == q.QAOA_ERR_INVALID_ARG
    assert q.lib.qaoa_xy_cost_vector(ct.byref(g), 2, None, q.COST_F64, ct.byref(desc), None) == q.QAOA_ERR_INVALID_ARG
    big = q.Graph(41, np.array([[0, 40]]), None).as_struct()
    assert q.lib.qaoa_xy_cost_vector(ct.byref(big), 2, fake, q.COST_I32, ct.byref(desc), None) == q.QAOA_ERR_INVALID_ARG
    rep = q.Graph(36, np.array([[0, 35], [35, 0]]), None).as_struct()
    assert q.lib.qaoa_xy_cost_vector(ct.byref(rep), 2, fake, q.COST_I32, ct.byref(desc), None) == q.QAOA_ERR_INVALID_ARG
    cost = q.CostT(1 << 21, q.COST_I32, 0, 10)
    gm = (ct.c_double * 2)(0.1, 0.2)
    bt = (ct.c_double * 2)(0.3, float("nan"))
    ok_b = (ct.c_double * 2)(0.3, 0.4)
    args = lambda n, k, dt, psi, c, b, ws, wsb: q.lib.qaoa_xy_apply_layers(n, k, dt, psi, c, gm, b, 2, 1, None, ws, wsb, None)
    E = q.QAOA_ERR_INVALID_ARG
    assert args(10, 11, q.C128, fake, ct.byref(cost), ok_b, fake, 1 << 20) == E      # k > n
    assert args(10, 5, 9, fake, ct.byref(cost), ok_b, fake, 1 << 20) == E            # dtype
    assert args(10, 5, q.C128, None, ct.byref(cost), ok_b, fake, 1 << 20) == E       # no state
    assert args(10, 5, q.C128, fake, None, ok_b, fake, 1 << 20) == E                 # no cost
    assert args(10, 5, q.C128, fake, ct.byref(cost), bt, fake, 1 << 20) == E         # non-finite angle
    assert args(10, 5, q.C128, fake, ct.byref(cost), ok_b, ct.c_void_p((1 << 20) + 8), 1 << 20) == E  # misaligned
    assert args(10, 5, q.C128, fake, ct.byref(cost), ok_b, fake, 256) == q.QAOA_ERR_WORKSPACE
    out = ct.c_void_p(1 << 22)
    assert q.lib.qaoa_xy_expectation(10, 5, q.C64, fake, ct.byref(cost), out, fake, 16, None) == q.QAOA_ERR_WORKSPACE
    assert q.lib.qaoa_xy_expectation(10, 5, q.C64, fake, ct.byref(cost), None, fake, 1 << 20, None) == E


def test_xy_gradient_rejects_bad_arguments_before_launch():
    fake, other = ct.c_void_p(1 << 20), ct.c_void_p(1 << 24)  # never dereferenced
    cost = q.CostT(1 << 21, q.COST_I32, 0, 10)
    gm = (ct.c_double * 2)(0.1, 0.2)
    ok_b = (ct.c_double * 2)(0.3, 0.4)
    bad_b = (ct.c_double * 2)(0.3, float("inf"))
    out = ct.c_void_p(1 << 22)
    need = ct.c_size_t()
    assert q.lib.qaoa_xy_gradient_workspace_size(10, 5, q.C128, 2, 11, ct.byref(need)) == q.QAOA_OK
    assert need.value > 0
    E = q.QAOA_ERR_INVALID_ARG
    call = lambda n, k, psi, lam, c, b, o, ws, wsb: q.lib.qaoa_xy_gradient(n, k, q.C128, psi, lam, c, gm, b, 2, o, ws,
                                                                           wsb, None)
    assert call(10, 5, fake, fake, ct.byref(cost), ok_b, out, fake, need.value) == E       # psi == lambda
    assert call(10, 5, fake, None, ct.byref(cost), ok_b, out, fake, need.value) == E       # no lambda
    assert call(10, 5, fake, other, ct.byref(cost), ok_b, None, fake, need.value) == E     # no output
    assert call(10, 5, fake, other, None, ok_b, out, fake, need.value) == E                # no cost
    assert call(10, 11, fake, other, ct.byref(cost), ok_b, out, fake, need.value) == E     # k > n
    assert call(10, 5, fake, other, ct.byref(cost), bad_b, out, fake, need.value) == E     # non-finite angle
    assert call(10, 5, fake, other, ct.byref(cost), ok_b, out, ct.c_void_p((1 << 20) + 8), need.value) == E
    assert call(10, 5, fake, other, ct.byref(cost), ok_b, out, fake, need.value - 1) == q.QAOA_ERR_WORKSPACE


def test_xy_sample_rejects_bad_arguments_before_launch():
    fake = ct.c_void_p(1 << 20)
    cost = q.CostT(1 << 21, q.COST_I32, 0, 10)
    need = ct.c_size_t()
    assert q.lib.qaoa_xy_sample_workspace_size(10, 5, ct.byref(need)) == q.QAOA_OK and need.value > 0
    assert q.lib.qaoa_xy_sample_workspace_size(10, 11, ct.byref(need)) == q.QAOA_ERR_INVALID_ARG
    E = q.QAOA_ERR_INVALID_ARG
    s = lambda n, k, dt, psi, c, shots, z, ws, wsb: q.lib.qaoa_xy_sample(n, k, dt, psi, c, shots, 1, z, z, ws, wsb, None)
    assert s(10, 5, q.C128, None, ct.byref(cost), 10, fake, fake, 1 << 20) == E           # no state
    assert s(10, 5, q.C128, fake, None, 10, fake, fake, 1 << 20) == E                     # no cost
    assert s(10, 5, q.C128, fake, ct.byref(cost), -1, fake, fake, 1 << 20) == E           # negative shots
    assert s(10, 5, q.C128, fake, ct.byref(cost), 10, None, fake, 1 << 20) == E           # no output
    assert s(10, 5, 7, fake, ct.byref(cost), 10, fake, fake, 1 << 20) == E                # dtype
    assert s(10, 5, q.C128, fake, ct.byref(cost), 10, fake, ct.c_void_p((1 << 20) + 8), 1 << 20) == E
    assert s(10, 5, q.C128, fake, ct.byref(cost), 10, fake, fake, 16) == q.QAOA_ERR_WORKSPACE


def test_xy_binding_checks_buffer_sizes_first():
    torch = pytest.importorskip("torch")
    cv = q.CostVector(torch.zeros(q.xy_dim(10, 5), dtype=torch.int32), 10)
    short = torch.zeros(q.xy_dim(10, 5) - 1, dtype=torch.complex128)
    with pytest.raises(ValueError):
        q.xy_apply_layers(short, 10, 5, cv, [0.1], [0.2])
    with pytest.raises(ValueError):
        q.xy_expectation(torch.zeros(q.xy_dim(10, 4), dtype=torch.complex128), 10, 5, cv)


def test_binding_checks_state_and_cost_sizes():
    torch = pytest.importorskip("torch")
    cv = q.CostVector(torch.zeros(1 << 10, dtype=torch.int32), 10)
    assert q._state_qubits(torch.zeros(1 << 10, dtype=torch.complex128), cv) == 10
    for bad in (1000, 1, 1 << 11):
        with pytest.raises(ValueError):
            q._state_qubits(torch.zeros(bad, dtype=torch.complex128), cv)
    with pytest.raises(ValueError):  # second state of another size
        q._state_qubits(torch.zeros(1 << 10, dtype=torch.complex128), cv, torch.zeros(1 << 9, dtype=torch.complex128))


def test_binding_checks_cost_vector_out_buffers():
    torch = pytest.importorskip("torch")
    g = q.Graph(6, np.array([[0, 1], [1, 2]]), None, True)
    for bad in (torch.zeros(63, dtype=torch.int32), torch.zeros(64, dtype=torch.float64),
                torch.zeros(128, dtype=torch.int32)[::2]):
        with pytest.raises(ValueError):
            q.cost_vector(g, "i32", out=bad)
    with pytest.raises(ValueError):
        q.cost_vector_pubo(6, [1], [1.0], out=torch.zeros(32, dtype=torch.int32))
    with pytest.raises(ValueError):
        q.xy_cost_vector(g, 3, out=torch.zeros(q.xy_dim(6, 3) + 1, dtype=torch.int32))


def test_binding_checks_layout_and_cost_dtype():
    torch = pytest.importorskip("torch")
    psi = torch.zeros(1 << 10, dtype=torch.complex128)
    with pytest.raises(ValueError):  # float32 costs would be read as float64
        q._state_qubits(psi, q.CostVector(torch.zeros(1 << 10, dtype=torch.float32), 10))
    cv = q.CostVector(torch.zeros(1 << 10, dtype=torch.float64), 10)
    assert q._state_qubits(psi, cv) == 10
    with pytest.raises(ValueError):  # strided view
        q._state_qubits(torch.zeros(1 << 11, dtype=torch.complex128)[::2], cv)


def test_binding_checks_optimizer_buffers():
    torch = pytest.importorskip("torch")
    cv = q.CostVector(torch.zeros(1 << 8, dtype=torch.float64), 8)
    ang = torch.zeros(6, dtype=torch.float64)
    st_size = ct.c_size_t()
    assert q.lib.qaoa_optimizer_state_size(q.OPTIMIZER_LBFGS, 3, ct.byref(st_size)) == 0
    q._check_optimizer_args("lbfgs", cv, ang, torch.zeros(st_size.value // 8, dtype=torch.float64))
    for bad_ang in (torch.zeros(6, dtype=torch.float32), torch.zeros(5, dtype=torch.float64),
                    torch.zeros(12, dtype=torch.float64)[::2]):
        with pytest.raises(ValueError):
            q._check_optimizer_args("adam", cv, bad_ang, None)
    with pytest.raises(ValueError):  # state too short for p = 3
        q._check_optimizer_args("lbfgs", cv, ang, torch.zeros(st_size.value // 8 - 1, dtype=torch.float64))
    with pytest.raises(ValueError):  # cost vector of the wrong length for n
        q._check_optimizer_args("adam", q.CostVector(torch.zeros(100, dtype=torch.int32), 8), ang, None)
