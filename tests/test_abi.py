"""The C-ABI library loads, exports every entry point include/rplu.h declares,
and rejects bad arguments before touching the GPU (runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rp():
    from paper_2601_22344_gb300.build import build_library
    build_library()
    import paper_2601_22344_gb300 as rp
    return rp


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rplu_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(rp):
    decl = _declared()
    assert {"rplu_dense", "rplu_cauchy", "rplu_batch"} <= set(decl)
    lib = ctypes.CDLL(rp.binding.LIB_PATH)
    for name in decl:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(rp.EXPORTED) <= set(decl)


def test_status_strings_and_version(rp):
    assert rp.status_string(rp.RPLU_OK) == "ok"
    assert "invalid" in rp.status_string(rp.RPLU_ERR_INVALID)
    assert rp.version() >= 100


def test_struct_layouts_match_header(rp, tmp_path):
    """The ctypes mirrors of rplu_opts and rplu_job have the header's layout
    (sizes and field offsets as compiled by gcc from include/rplu.h)."""
    o = rp.Opts()
    rp.lib.rplu_opts_init(ctypes.byref(o))
    assert o.dtype == 1 and o.pivot == 0 and o.rel_tol == 0.0 and o.stream is None
    lines = []
    for cname, py in (("rplu_opts", rp.Opts), ("rplu_job", rp.Job)):
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "rplu.h"\nint main(void) {\n'
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for py in (rp.Opts, rp.Job):
        want.append(ctypes.sizeof(py))
        want += [getattr(py, f).offset for f, _ in py._fields_]
    assert got == want


def _call_dense(rp, n, m, k, opts=None, A=True, outs=True):
    a = np.zeros((max(n, 1), max(m, 1))) if A else None
    I = np.zeros(max(k, 1), np.int64)
    L = np.zeros(max(n * k, 1))
    U = np.zeros(max(k * m, 1))
    kd = ctypes.c_int64(-7)
    o = opts or rp.Opts()
    if opts is None:
        rp.lib.rplu_opts_init(ctypes.byref(o))
    return rp.lib.rplu_dense(a.ctypes.data if A else None, n, m, k, 0, ctypes.byref(o),
                             I.ctypes.data if outs else None, I.ctypes.data if outs else None,
                             L.ctypes.data if outs else None, U.ctypes.data if outs else None, ctypes.byref(kd))


def test_invalid_arguments_rejected_on_host(rp):
    assert _call_dense(rp, 5, 4, 5) == rp.RPLU_ERR_INVALID           # k > min(n, m)
    assert _call_dense(rp, -1, 4, 0) == rp.RPLU_ERR_INVALID          # negative size
    assert _call_dense(rp, 5, 4, 2, outs=False) == rp.RPLU_ERR_INVALID
    assert _call_dense(rp, 5, 4, 2, A=False) == rp.RPLU_ERR_INVALID
    o = rp.Opts()
    rp.lib.rplu_opts_init(ctypes.byref(o))
    o.dtype = 9
    assert _call_dense(rp, 5, 4, 2, opts=o) == rp.RPLU_ERR_INVALID
    o.dtype = 1
    o.rel_tol = -1.0
    assert _call_dense(rp, 5, 4, 2, opts=o) == rp.RPLU_ERR_INVALID
    o.rel_tol = 0.0
    o.pivot = 3  # given pivots without arrays
    assert _call_dense(rp, 5, 4, 2, opts=o) == rp.RPLU_ERR_INVALID
    assert rp.lib.rplu_dense(None, 1, 1, 0, 0, None, None, None, None, None, None) == rp.RPLU_ERR_INVALID
    assert b"k_done" in rp.lib.rplu_last_error()
    o.pivot = 2
    o.rel_tol = 0.1  # complete pivoting takes no tolerance
    assert _call_dense(rp, 5, 4, 2, opts=o) == rp.RPLU_ERR_INVALID
    x = np.zeros(3, np.complex128)
    kd = ctypes.c_int64(0)
    o2 = rp.Opts()
    rp.lib.rplu_opts_init(ctypes.byref(o2))
    o2.pivot = 2
    o2.dtype = 3
    assert rp.lib.rplu_cauchy(x.ctypes.data, x.ctypes.data, 3, 3, 1, 0, ctypes.byref(o2), x.ctypes.data,
                              x.ctypes.data, x.ctypes.data, x.ctypes.data, ctypes.byref(kd)) == rp.RPLU_ERR_INVALID


def _opts(rp, **kw):
    o = rp.Opts()
    rp.lib.rplu_opts_init(ctypes.byref(o))
    for k_, v in kw.items():
        setattr(o, k_, v)
    return o


def test_newer_entry_points_reject_bad_arguments_on_host(rp):
    """Argument checks of the Cauchy-like (with and without bounds), bounds,
    plan-size, CUR-form, CUR-AAA and barycentric entry points run before any
    CUDA call, so they answer RPLU_ERR_INVALID with a message on a machine
    without a GPU."""
    lib, INV = rp.lib, rp.RPLU_ERR_INVALID
    x = np.zeros(8, np.complex128)
    G = np.zeros(64, np.complex128)
    i64 = np.zeros(8, np.int64)
    kd = ctypes.c_int64(0)
    p = x.ctypes.data

    def cl(o, pp=1, k=2):
        return lib.rplu_cauchy_like(p, p, G.ctypes.data, G.ctypes.data, 8, 8, pp, k, 0, ctypes.byref(o),
                                    i64.ctypes.data, i64.ctypes.data, p, p, ctypes.byref(kd))

    def msg():
        return lib.rplu_last_error().decode()

    assert cl(_opts(rp, dtype=3), pp=5) == INV and "displacement rank" in msg()
    assert cl(_opts(rp, dtype=3, pivot=2)) == INV and "dense form" in msg()
    assert cl(_opts(rp, dtype=3, bound_nu=0.5)) == INV and "bound_nu" in msg()
    assert cl(_opts(rp, dtype=3, bound_nu=float("inf"))) == INV and "bound_nu" in msg()
    assert cl(_opts(rp, dtype=3, bound_nu=5.0, bound_stop=2)) == INV and "bound_stop" in msg()
    assert cl(_opts(rp, dtype=3, bound_nu=5.0, bound_leaf=-1)) == INV and "bound_leaf" in msg()
    assert cl(_opts(rp, dtype=3, bound_nu=5.0, pivot=3, given_I=i64.ctypes.data, given_J=i64.ctypes.data)) == INV
    assert "RANDOM or RPLU_PIVOT_C2" in msg()
    assert cl(_opts(rp, dtype=3), k=9) == INV and "k exceeds" in msg()

    u = np.zeros(8)
    o = _opts(rp, dtype=3)
    bb = lib.rplu_bh_bounds
    assert bb(p, p, G.ctypes.data, G.ctypes.data, 0, 8, 1, 5.0, 32, ctypes.byref(o), u.ctypes.data) == INV
    assert bb(p, p, G.ctypes.data, G.ctypes.data, 8, 8, 1, 0.9, 32, ctypes.byref(o), u.ctypes.data) == INV
    assert bb(p, p, G.ctypes.data, G.ctypes.data, 8, 8, 1, 5.0, 0, ctypes.byref(o), u.ctypes.data) == INV
    assert "leaf size" in msg()
    assert bb(p, p, G.ctypes.data, G.ctypes.data, 8, 8, 1, 5.0, 32, ctypes.byref(o), None) == INV
    st = np.zeros(6, np.int64)
    ps = lib.rplu_bh_plan_stats
    assert ps(p, p, 8, 8, float("nan"), 32, ctypes.byref(o), st.ctypes.data) == INV
    assert ps(p, p, 8, 8, 5.0, 32, ctypes.byref(o), None) == INV and "NULL" in msg()

    cur = lib.rplu_cauchy_cur
    assert cur(p, p, 8, 8, 2, 0, ctypes.byref(_opts(rp, dtype=3, pivot=2)), i64.ctypes.data, i64.ctypes.data,
               G.ctypes.data, ctypes.byref(kd)) == INV and "dense form" in msg()
    assert cur(None, p, 8, 8, 2, 0, ctypes.byref(o), i64.ctypes.data, i64.ctypes.data, G.ctypes.data,
               ctypes.byref(kd)) == INV and "NULL" in msg()

    kk = ctypes.c_int64(0)
    which = ctypes.c_int32(0)
    err = np.zeros(2)

    def aaa(o, m=8, eps=1e-8, k_max=4):
        return lib.rplu_cur_aaa(p, p, m, eps, k_max, 0, ctypes.byref(o), i64.ctypes.data, G.ctypes.data,
                                ctypes.byref(kk), ctypes.byref(which), err.ctypes.data)

    assert aaa(_opts(rp, dtype=2)) == INV and "RPLU_C128" in msg()
    assert aaa(_opts(rp, dtype=3, pivot=2)) == INV
    assert aaa(_opts(rp, dtype=3), m=1) == INV and "m must be" in msg()
    assert aaa(_opts(rp, dtype=3), eps=0.0) == INV and "eps" in msg()
    assert aaa(_opts(rp, dtype=3), k_max=0) == INV and "k_max" in msg()

    bary = lib.rplu_barycentric
    assert bary(p, p, p, 0, p, 4, ctypes.byref(o), p) == INV and "k must be" in msg()
    assert bary(p, p, p, 2, None, 4, ctypes.byref(o), p) == INV and "NULL" in msg()


def test_toeplitz3_cur_rejects_bad_arguments_on_host(rp):
    lib, INV = rp.lib, rp.RPLU_ERR_INVALID
    I = np.zeros(8, np.int64)
    C = np.zeros(64)
    kd = ctypes.c_int64(0)

    def call(N=4, length=320.0, delta=50.0, sigma=80.0, k=2, o=None, kd_=True):
        o = o or _opts(rp)
        return lib.rplu_toeplitz3_cur(N, length, delta, sigma, k, 0, ctypes.byref(o), I.ctypes.data, I.ctypes.data,
                                      C.ctypes.data, ctypes.byref(kd) if kd_ else None)

    assert call(N=0) == INV and "N must be" in lib.rplu_last_error().decode()
    assert call(N=641) == INV
    assert call(sigma=0.0) == INV and call(length=float("inf")) == INV and call(delta=float("nan")) == INV
    assert call(N=2, k=9) == INV and "k must be" in lib.rplu_last_error().decode()
    assert call(kd_=False) == INV
    assert call(o=_opts(rp, pivot=2)) == INV
    assert call(o=_opts(rp, pivot=3)) == INV and "given" in lib.rplu_last_error().decode()
    assert call(o=_opts(rp, rel_tol=-1.0)) == INV


def test_sparse_cur_rejects_malformed_csr_on_host(rp):
    lib, INV = rp.lib, rp.RPLU_ERR_INVALID
    out_I = np.zeros(4, np.int64)
    C = np.zeros(16)
    kd = ctypes.c_int64(0)

    def call(rp_, ci, v, n=3, m=3, k=2, o=None):
        rp_ = np.asarray(rp_, np.int64)
        ci = np.asarray(ci, np.int32)
        v = np.asarray(v, np.float64)
        o = o or _opts(rp)
        st = lib.rplu_sparse_cur(n, m, rp_.ctypes.data, ci.ctypes.data, v.ctypes.data, k, 0, ctypes.byref(o),
                                 out_I.ctypes.data, out_I.ctypes.data, C.ctypes.data, ctypes.byref(kd))
        return st, lib.rplu_last_error().decode()

    good = ([0, 2, 3, 4], [0, 2, 1, 0], [1.0, 2.0, 3.0, 4.0])
    assert call([1, 2, 3, 4], good[1], good[2]) == (INV, "row_ptr[0] must be 0")
    assert call([0, 3, 2, 4], good[1], good[2])[1] == "row_ptr must be nondecreasing"
    assert call(good[0], [0, 3, 1, 0], good[2])[1] == "column index out of range"
    assert call(good[0], [2, 0, 1, 0], good[2])[1].startswith("column indices must increase")
    assert call(good[0], [1, 1, 1, 0], good[2])[1].startswith("column indices must increase")  # a duplicate
    assert call(good[0], good[1], [1.0, np.inf, 3.0, 4.0])[1] == "input has a non-finite entry"
    assert call(good[0], good[1], good[2], k=4)[0] == INV
    assert call(good[0], good[1], good[2], n=0)[0] == INV
    assert call(good[0], good[1], good[2], o=_opts(rp, pivot=2))[0] == INV


def test_no_cpu_fallback_without_a_gpu(rp):
    """Without a usable GPU every compute entry point fails loudly (RPLU_ERR_CUDA
    through the binding as RPLUError); nothing is computed on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import scipy.sparse as sp
    A = np.random.default_rng(0).standard_normal((40, 30))
    x = np.linspace(0.0, 1.0, 30) + 0j
    y = np.linspace(3.0, 4.0, 20) + 0j
    calls = [
        lambda: rp.rplu_dense(A, 5),
        lambda: rp.rplu_cauchy(x, y, 5),
        lambda: rp.rplu_cauchy_cur(x, y, 5),
        lambda: rp.rplu_cauchy_like(x, y, np.ones((30, 1), complex), np.ones((1, 20), complex), 5),
        lambda: rp.rplu_toeplitz3_cur(4, 5, device="host"),
        lambda: rp.rplu_sparse_cur(sp.random(30, 20, density=0.2, random_state=1), 5, device="host"),
        lambda: rp.rplu_cur_aaa(x, np.tan(x), eps=1e-8),
    ]
    for call in calls:
        with pytest.raises(rp.RPLUError) as e:
            call()
        assert e.value.status == rp.RPLU_ERR_CUDA


def test_vectorized_host_cauchy_job_table_equals_the_generic_one(rp):
    """The host-Cauchy marshalling path writes the same job table as the
    per-job one (sizes, k_max, tolerance, per-job seeds), with pointers into
    packed copies of the same points."""
    import workloads as W
    import paper_2601_22344_gb300.batch as B
    from paper_2601_22344_gb300.binding import Job
    blocks = W.cauchy_interval_blocks(7, seed=3, size_lo=5, size_hi=90)
    specs = [dict(kind="cauchy", x=b.x, y=b.y, dtype="f32") for b in blocks]
    assert B._host_cauchy_uniform(specs) == "f32"
    a1, a2 = (Job * 7)(), (Job * 7)()
    B._fill(a1, specs, 1e-6, 11, None)
    keep, packed = B._fill_host_cauchy(a2, specs, "f32", 1e-6, 11, None)
    for b in range(7):
        for name, _ in Job._fields_:
            if name in ("x", "y", "I", "J", "L", "U"):
                continue
            assert getattr(a1[b], name) == getattr(a2[b], name), (b, name)
        x = np.ctypeslib.as_array(ctypes.cast(a2[b].x, ctypes.POINTER(ctypes.c_float)), (a2[b].n,))
        y = np.ctypeslib.as_array(ctypes.cast(a2[b].y, ctypes.POINTER(ctypes.c_float)), (a2[b].m,))
        assert np.array_equal(x, blocks[b].x.astype(np.float32)) and np.array_equal(y, blocks[b].y.astype(np.float32))
    mixed = specs[:2] + [dict(kind="dense", A=np.ones((3, 3)), dtype="f32")]
    assert B._host_cauchy_uniform(mixed) is None


def test_packed_range_job_table_equals_the_per_spec_one(rp):
    """rplu_batch_cauchy_packed's job table (points as consecutive ranges of two
    arrays) equals the one built from per-job specs of the same points, and
    sizes that do not add up are refused before any call."""
    import workloads as W
    import paper_2601_22344_gb300.batch as B
    from paper_2601_22344_gb300.binding import Job
    blocks = W.cauchy_interval_blocks(9, seed=5, size_lo=5, size_hi=90)
    specs = [dict(kind="cauchy", x=b.x, y=b.y, dtype="f32") for b in blocks]
    X = np.concatenate([b.x for b in blocks]).astype(np.float32)
    Y = np.concatenate([b.y for b in blocks]).astype(np.float32)
    n = np.array([len(b.x) for b in blocks])
    m = np.array([len(b.y) for b in blocks])
    a1, a2 = (Job * 9)(), (Job * 9)()
    B._fill_host_cauchy(a1, specs, "f32", 1e-6, 11, 7)
    keep, packed = B._fill_packed(a2, X, Y, n, m, "f32", 1e-6, 11, 7)
    for b in range(9):
        for name, _ in Job._fields_:
            if name in ("x", "y", "I", "J", "L", "U"):
                continue
            assert getattr(a1[b], name) == getattr(a2[b], name), (b, name)
        x = np.ctypeslib.as_array(ctypes.cast(a2[b].x, ctypes.POINTER(ctypes.c_float)), (a2[b].n,))
        assert np.array_equal(x, blocks[b].x.astype(np.float32))
    with pytest.raises(ValueError):
        B.rplu_batch_cauchy_packed(X, Y, n[:-1], m[:-1])


def test_packed_range_outputs_reused_only_for_the_same_jobs(rp):
    """out= writes into an earlier call's packed output arrays: the job
    table's output pointers are those of the earlier table, and outputs of
    other sizes, k_max or dtype are refused before any call."""
    import workloads as W
    import paper_2601_22344_gb300.batch as B
    from paper_2601_22344_gb300.binding import Job
    blocks = W.cauchy_interval_blocks(6, seed=9, size_lo=5, size_hi=70)
    X = np.concatenate([b.x for b in blocks]).astype(np.float32)
    Y = np.concatenate([b.y for b in blocks]).astype(np.float32)
    n = np.array([len(b.x) for b in blocks])
    m = np.array([len(b.y) for b in blocks])
    a1, a2 = (Job * 6)(), (Job * 6)()
    _, packed = B._fill_packed(a1, X, Y, n, m, "f32", 1e-6, 3, None)
    prev = B.PackedResults(a1, packed, 6)
    _, again = B._fill_packed(a2, X, Y, n, m, "f32", 1e-6, 4, None, prev)
    assert all(again[q] is packed[q] for q in range(4))
    for b in range(6):
        assert (a1[b].I, a1[b].J, a1[b].L, a1[b].U) == (a2[b].I, a2[b].J, a2[b].L, a2[b].U)
        assert a1[b].seed != a2[b].seed
        assert (a1[b].memory, a2[b].memory) == (1, 3)  # reused outputs: written in place where possible
    m2 = m.copy()
    m2[0] += 1
    for bad in (dict(m=m2, dt="f32", k_max=None), dict(m=m, dt="f32", k_max=4), dict(m=m, dt="f64", k_max=None)):
        with pytest.raises(ValueError):
            B._fill_packed((Job * 6)(), X, Y, n, bad["m"], bad["dt"], 1e-6, 3, bad["k_max"], prev)
    with pytest.raises(TypeError):
        B.rplu_batch_cauchy_packed(X, Y, n, m, out=packed)


def test_session_options_checked_before_any_device_call(rp):
    """Session defaults, and malformed session options (bound_nu in (0, 1)
    or not finite, sizes above the kernel's 4096) refused before the device
    is touched."""
    from paper_2601_22344_gb300 import serve as S
    from paper_2601_22344_gb300.binding import SessionOpts, lib
    o = SessionOpts()
    lib.rplu_session_opts_init(ctypes.byref(o))
    assert (o.max_jobs, o.max_dim, o.idle_us, o.large_streams, o.cauchy_max_dim, o.bound_nu) == \
        (4096, 2048, 1000.0, 8, 0, 0.0)
    for bad in (dict(bound_nu=0.5), dict(bound_nu=float("nan")), dict(bound_nu=float("inf")),
                dict(max_dim=5000), dict(cauchy_max_dim=5000), dict(large_streams=65)):
        with pytest.raises(rp.RPLUError) as e:
            S.Session(**bad)
        assert e.value.status == rp.RPLU_ERR_INVALID, bad
