"""The C ABI library loads on a machine without a GPU, exports every symbol that
include/oed.h declares, and its host-only entry points behave (no kernel runs)."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    import paper_1502_07873_gb300 as P
    return P


def _declared():
    src = open(os.path.join(ROOT, "include", "oed.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(oed_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported(P):
    L = P.library()
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(P.SYMBOLS)


def test_status_strings(P):
    L = P.library()
    assert L.oed_status_string(0) == b"OED_OK"
    assert L.oed_status_string(3) == b"OED_ENOTPD"
    assert L.oed_status_string(99) == b"unknown"


def test_workspace_bytes(P):
    w = W.batched()
    p = P.problem_from_workload(w, P.OED_FP32)
    b = P.oed_workspace_bytes(p, 3840)
    xp = 416
    field = 3840 * 2 * w.nz * xp * 4
    assert 2 * field < b < 2 * field * 1.3
    p64 = P.problem_from_workload(w, P.OED_FP64)
    assert P.oed_workspace_bytes(p64, 3840) > 1.9 * b
    bad = P.make_problem(4, 4, 1.0, 1e-3, 10, W.HOMOGENEOUS, [0])
    assert P.oed_workspace_bytes(bad, 100) == 0
    bad2 = P.problem_from_workload(w, P.OED_FP32, rec_ix=[w.nx])
    assert P.oed_workspace_bytes(bad2, 100) == 0


def test_create_rejects_bad_problem_without_touching_the_device(P):
    L = P.library()
    h = ctypes.c_void_p()
    bad = P.make_problem(401, 201, -5.0, 1e-3, 10, W.HOMOGENEOUS, [3])
    assert L.oed_create(ctypes.byref(h), ctypes.byref(bad), 100) == P.OED_EINVAL
    assert not h.value
    assert L.oed_destroy(None) == P.OED_OK


@pytest.mark.parametrize("dim,level", [(3, 5), (7, 3), (2, 9), (7, 5)])
def test_smolyak_host_matches_oracle(P, oracle, dim, level):
    x, w = P.oed_nodes_smolyak(dim, level)
    xo, wo = oracle.smolyak(dim, level)
    assert x.shape == xo.shape
    assert np.max(np.abs(x - xo)) < 1e-13
    assert np.max(np.abs(w - wo)) < 1e-11
    lo = np.array(W.PRIOR_LO)[:dim]
    hi = np.array(W.PRIOR_HI)[:dim]
    xm, wm = P.oed_nodes_smolyak(dim, level, lo, hi)
    assert np.allclose(xm, lo + (hi - lo) * (xo + 1) / 2, rtol=1e-13)


def test_smolyak_host_rejects_small_buffer(P):
    L = P.library()
    cnt = ctypes.c_int()
    x = np.zeros((10, 7))
    wt = np.zeros(10)
    rc = L.oed_nodes_smolyak(7, 3, None, None, 10, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             wt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(cnt))
    assert rc == P.OED_ENOMEM and cnt.value == 589


def test_product_path_has_no_oracle_import():
    """The package must not reach the oracle (or any CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_1502_07873_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.replace("the oracle", ""), f


def test_time_function_kind_is_validated_on_the_host(P):
    """stf must be Gaussian or Ricker; the server refuses sensitivity solves with a Ricker
    source at submission (request bytes 0), before any device work."""
    w = W.batched()
    gauss = P.oed_workspace_bytes(P.problem_from_workload(w), 100)
    assert gauss > 0
    assert P.oed_workspace_bytes(P.problem_from_workload(w, stf=P.OED_STF_RICKER), 100) == gauss
    assert P.oed_workspace_bytes(P.problem_from_workload(w, stf=2), 100) == 0
    assert P.oed_workspace_bytes(P.problem_from_workload(w, stf=-1), 100) == 0
    L = P.library()
    p = P.problem_from_workload(w, stf=P.OED_STF_RICKER)
    th = np.tile(np.array(w.prior_lo) * 0.5 + np.array(w.prior_hi) * 0.5, (4, 1))
    sizes = {}
    for jac in (P.OED_JAC_PAIRS, P.OED_JAC_DIFFERENCE, P.OED_JAC_SENSITIVITY):
        req = P.make_request(p, th, np.full(4, 0.25), w.prior_lo, w.prior_hi, w.rel_step, 0.1, jac)
        sizes[jac] = L.oed_server_request_bytes(ctypes.byref(req), 16)
    assert sizes[P.OED_JAC_PAIRS] > sizes[P.OED_JAC_DIFFERENCE] > 0
    assert sizes[P.OED_JAC_SENSITIVITY] == 0


_CTYPE_OF = {"int": ctypes.c_int, "double": ctypes.c_double, "size_t": ctypes.c_size_t,
             "unsigned long long": ctypes.c_ulonglong, "unsigned int": ctypes.c_uint,
             "unsigned": ctypes.c_uint}


def _prototypes():
    src = open(os.path.join(ROOT, "include", "oed.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"#[^\n]*", "", src)
    out = {}
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(oed_[a-z_]+)\s*\(([^)]*)\)\s*;", src):
        params = [p.strip() for p in m.group(3).split(",")]
        out[m.group(2)] = [] if params == ["void"] or params == [""] else params
    return out


def test_binding_argument_types_match_the_header(P):
    """Every prototype of include/oed.h and the binding's argtypes agree in arity and in
    kind: pointers for pointer parameters, int / double / size_t for the scalars."""
    L = P.library()
    protos = _prototypes()
    assert set(protos) == set(P.SYMBOLS)
    for name, params in protos.items():
        argtypes = getattr(L, name).argtypes
        assert len(argtypes) == len(params), (name, params, argtypes)
        for p, t in zip(params, argtypes):
            if "*" in p:
                assert t is ctypes.c_void_p or t is ctypes.c_char_p or hasattr(t, "contents") or \
                    issubclass(t, ctypes._Pointer), (name, p, t)
            else:
                words = p.replace("const", "").split()[:-1]   # the type, without the name
                assert t is _CTYPE_OF[" ".join(words)], (name, p, t)


def test_struct_mirrors_match_the_c_layout(P, tmp_path):
    """The ctypes mirrors of oed_problem, oed_request and oed_result have the C sizes and
    field offsets (compiled and measured with the host C compiler)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"oed_problem": P.Problem, "oed_request": P.Request, "oed_result": P.Result}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "oed.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n"):
        if line:
            s, f, v = line.split()
            got[(s, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_workspace_holds_two_level_pairs_off_chip(P):
    """FP32 grids that do not fit on chip reserve a second pair of levels (the two-step
    kernel reads one pair and writes the other); FP32 grids that fit, and FP64, do not."""
    w = W.layered()                     # 801x401: does not fit on chip
    n = 700
    level32 = n * 2 * w.nz * 832 * 4    # one FP32 level (two components, padded rows)
    f32 = P.oed_workspace_bytes(P.problem_from_workload(w, P.OED_FP32), n)
    f64 = P.oed_workspace_bytes(P.problem_from_workload(w, P.OED_FP64), n)
    assert 4 * level32 < f32 < 4 * level32 * 1.2
    assert 4 * level32 < f64 < 4 * level32 * 1.3   # two FP64 levels (and 8-byte traces)
    b = W.batched()                     # 401x201 fits on chip: one pair
    fb = P.oed_workspace_bytes(P.problem_from_workload(b, P.OED_FP32), n)
    assert 2 * n * 2 * b.nz * 416 * 4 < fb < 3 * n * 2 * b.nz * 416 * 4


def test_workspace_holds_the_paired_layout(P):
    """The two-step kernel keeps its levels in the paired layout: per row the even columns'
    (x, z) pairs in sq slots, then the odd columns', sq = (nx + 1) / 2 + 4 rounded up to
    even.  At 415 columns that is 848 floats a row against the planar 2 x 416, so the
    workspace reserves the larger per solve."""
    w = W.tiny(nx=415, nz=801, h=5.0, nsteps=50, nrec=4)
    n = 30
    sq = ((415 + 1) // 2 + 4 + 1) & ~1
    paired_level = n * w.nz * 4 * sq * 4
    assert 4 * sq > 2 * 416
    f32 = P.oed_workspace_bytes(P.problem_from_workload(w, P.OED_FP32), n)
    assert f32 >= 4 * paired_level


def test_server_host_side_sizing_and_validation(P):
    """The server's footprint rule and submission checks run on the host: a request
    reserves a workspace for chunks of chunk_nodes nodes plus its arrays; a resume with
    more finished nodes than the request, or without their Hessians, is refused."""
    import numpy as np
    w = W.tiny(nx=61, nz=31, h=33.0, nsteps=40, nrec=3)
    n = 10
    rng = np.random.default_rng(3)
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    th = lo + (hi - lo) * rng.random((n, 7))
    prob = P.problem_from_workload(w, P.OED_FP32)
    r = P.make_request(prob, th, np.full(n, 0.1), w.prior_lo, w.prior_hi, w.rel_step, 0.1, P.OED_JAC_DIFFERENCE)
    L = P.library()
    b = L.oed_server_request_bytes(ctypes.byref(r), 4)
    assert b == P.oed_workspace_bytes(prob, 7 * 4) + n * 57 * 8 + 4096
    assert L.oed_server_request_bytes(ctypes.byref(r), 100) == P.oed_workspace_bytes(prob, 7 * n) + n * 57 * 8 + 4096
    with pytest.raises(ValueError):
        P.make_request(prob, th, np.full(n, 0.1), w.prior_lo, w.prior_hi, w.rel_step, 0.1, 1,
                       H_done=np.zeros((n + 1, 7, 7)))
    r.n_done = 3   # finished nodes without their Hessians
    rid = ctypes.c_ulonglong()
    assert L.oed_server_submit(None, ctypes.byref(r), ctypes.byref(rid)) == P.OED_EINVAL


def test_spread_sample_takes_both_ends_of_each_interval():
    """The node picker of the sampled checks: the given nodes first, then for x_s, z_s, t_s
    and omega_s the node nearest each end of its prior interval, without repeats."""
    import numpy as np
    w = W.batched()
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    th = lo + (hi - lo) * w.uniforms()
    idx = W.spread_sample(th, w.prior_lo, w.prior_hi)
    assert idx[:2] == [0, 1] and len(idx) == len(set(idx)) == 10
    u = (th - lo) / (hi - lo)
    for j in range(4):
        assert int(np.argmin(u[:, j])) in idx or np.argmin(u[:, j]) in (0, 1)
        assert int(np.argmax(u[:, j])) in idx or np.argmax(u[:, j]) in (0, 1)


def test_binding_checks_tensor_arguments_before_the_device(P):
    """The binding refuses a tensor of the wrong dtype, too few elements or the wrong
    parameter shape before anything reaches the library (such a tensor would be read or
    written past its end on the device); these calls need no context."""
    torch = pytest.importorskip("torch")
    lo, hi = W.PRIOR_LO, W.PRIOR_HI
    H = torch.zeros((2, 7, 7), dtype=torch.float64)
    w = torch.zeros(2, dtype=torch.float64)
    eig = torch.zeros(1, dtype=torch.float64)
    # each defect sits in the first tensor the call checks (the checks run argument by
    # argument; on a GPU every argument is a device tensor and all are checked)
    cases = [
        (lambda: P.oed_eig(None, H.float(), w, lo, hi, eig), "H: expected torch.float64"),
        (lambda: P.oed_eig(None, torch.zeros((2, 7, 6), dtype=torch.float64), w, lo, hi, eig),
         "H: needs at least 98"),
        (lambda: P.oed_nodes_mc(torch.zeros((3, 6), dtype=torch.float64), lo, hi,
                                torch.zeros((3, 7), dtype=torch.float64), torch.zeros(3, dtype=torch.float64)),
         "u: expected shape"),
        (lambda: P.oed_newton_step(H, torch.zeros((2, 7), dtype=torch.float64),
                                   torch.zeros((2, 6), dtype=torch.float64), lo, hi), "theta: expected shape"),
        (lambda: P.oed_dlmc(torch.zeros((4, 5), dtype=torch.float64), torch.zeros((3, 5), dtype=torch.float64),
                            torch.zeros((3, 5), dtype=torch.float64), 0.1, torch.zeros(4, dtype=torch.float64)),
         "shapes"),
        (lambda: P.oed_eig_designs(None, torch.zeros((2, 4, 1, 28), dtype=torch.float64), 0,
                                   torch.zeros((3, 5), dtype=torch.uint8), w, lo, hi, eig), "mask: expected shape"),
        # well-formed, but host tensors: refused as well, since the calls take device memory
        (lambda: P.oed_eig(None, H, w, lo, hi, eig), "expected a CUDA tensor"),
    ]
    for call, msg in cases:
        with pytest.raises(ValueError, match=msg):
            call()
