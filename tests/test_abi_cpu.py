"""The C ABI library on a machine without a GPU: it builds, loads, exports every function
include/sph.h declares, its structures match the ctypes mirrors byte for byte, and host-side
argument checks answer before any device work (no compute call runs here)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sph.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc is needed to build libsph.so")


@pytest.fixture(scope="module")
def B():
    from paper_1612_06090_gb300 import build, binding

    build.build()
    binding.lib()
    return binding


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_function(B):
    names = declared_functions()
    assert set(names) == set(B.EXPORTED)
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (sph_\w+)", out))
    for n in names:
        assert n in exported, n
        assert hasattr(B.lib(), n)


def test_probe_library_exports_its_header():
    """libsph_probe.so (the FP32 rate probe the bench divides by) exports what sph_probe.h
    declares."""
    from paper_1612_06090_gb300 import build

    build.build()
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "sph_probe.h")).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(sph_[a-z0-9_]+)\s*\(", text)))
    assert names == ["sph_probe_fp32_fma"]
    out = subprocess.run(["nm", "-D", "--defined-only", build.PROBE_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (sph_\w+)", out))
    assert set(names) <= exported
    lib = ctypes.CDLL(build.PROBE_PATH)
    tf, ms = ctypes.c_double(), ctypes.c_double()
    # argument checks answer before any device work
    assert lib.sph_probe_fp32_fma(None, 0, 10, 0, ctypes.byref(tf), ctypes.byref(ms)) == 1
    assert lib.sph_probe_fp32_fma(None, 8, 10, 0, None, ctypes.byref(ms)) == 1


def test_struct_layout_matches_header(tmp_path, B):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "sph.h"\n'
        "int main(void){\n"
        ' printf("%zu %zu %zu %zu %zu\\n", sizeof(sph_params), offsetof(sph_params, nngb),'
        " offsetof(sph_params, max_iter), offsetof(sph_params, tune_cache), sizeof(sph_stats));\n"
        ' printf("%zu %zu %zu\\n", offsetof(sph_stats, todo_per_pass), offsetof(sph_stats, pair_evals),'
        " offsetof(sph_stats, solve_ms));\n"
        ' printf("%zu %zu %zu\\n", sizeof(sph_tuning), offsetof(sph_tuning, item_cap),'
        " offsetof(sph_tuning, blocks_per_sm));\n return 0; }\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    a, b, c = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:3]
    P, S = B.SphParams, B.SphStats
    assert [int(v) for v in a.split()] == [ctypes.sizeof(P), P.nngb.offset, P.max_iter.offset,
                                           P.tune_cache.offset, ctypes.sizeof(S)]
    assert [int(v) for v in b.split()] == [S.todo_per_pass.offset, S.pair_evals.offset, S.solve_ms.offset]
    U = B.SphTuning
    assert [int(v) for v in c.split()] == [ctypes.sizeof(U), U.item_cap.offset, U.blocks_per_sm.offset]


def test_status_strings(B):
    for code in range(0, 9):
        s = B.sph_status_string(code)
        assert s and s != "unknown status"
    assert B.sph_status_string(99) == "unknown status"
    assert B.sph_last_error(None) == ""


def test_create_rejects_bad_arguments_on_the_host(B):
    good = B.make_params()
    L = B.lib()
    # NULL out pointer
    assert L.sph_create(ctypes.byref(good), 100, None, None) == B.SPH_ERR_INVALID_ARG
    # NULL params
    out = ctypes.c_void_p()
    assert L.sph_create(None, 100, None, ctypes.byref(out)) == B.SPH_ERR_INVALID_ARG
    cases = [
        dict(nngb=10.0),            # below the self term 32/3
        dict(nngb=float("nan")),
        dict(tol=-1.0),
        dict(max_iter=0),
        dict(max_iter=65),
        dict(box=(1.0, 0.0, 1.0)),
        dict(box=(1.0, float("inf"), 1.0)),
        dict(precision=7),
        dict(list_entries=8),       # cached lists hold 16..1024 entries
        dict(list_entries=2000),
        dict(list_entries=-1),
    ]
    for kw in cases:
        st, ctx = B.sph_create(B.make_params(**kw), 100)
        assert st == B.SPH_ERR_INVALID_ARG, kw
        assert ctx is None
    # Wendland C6's self term is 1365/48 = 28.4375: a target below it is rejected
    st, ctx = B.sph_create(B.make_params(kernel=B.SPH_KERNEL_WENDLAND_C6, nngb=20.0), 100)
    assert st == B.SPH_ERR_INVALID_ARG
    st, ctx = B.sph_create(B.make_params(kernel=7), 100)
    assert st == B.SPH_ERR_INVALID_ARG
    for cap in (0, -5, 1 << 31):
        st, ctx = B.sph_create(good, cap)
        assert st == B.SPH_ERR_INVALID_ARG


def test_calls_on_null_context(B):
    assert B.sph_sort(None, 10, 1, 1) == B.SPH_ERR_INVALID_ARG
    assert B.sph_density_solve(None, 1, 1, 1) == B.SPH_ERR_INVALID_ARG
    assert B.sph_density_eval(None, 1, 1, 1) == B.SPH_ERR_INVALID_ARG
    assert B.sph_batch_solve(None, 1, 1, 1, 1, 1, 1, 1, 1, 1) == B.SPH_ERR_INVALID_ARG
    assert B.sph_knn_solve(None, 64, 1, 1, 1) == B.SPH_ERR_INVALID_ARG
    assert B.sph_set_params(None, B.make_params()) == B.SPH_ERR_INVALID_ARG
    assert B.sph_interact(None, 1, 1, 1, 1, 1, 1, 1, 1) == B.SPH_ERR_INVALID_ARG
    B.sph_destroy(None)


def test_without_a_gpu_create_reports_cuda(B):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, ctx = B.sph_create(B.make_params(), 1000)
    assert st == B.SPH_ERR_CUDA
    assert ctx is None


def test_binding_rejects_tensors_the_library_would_misread(B):
    """The Solver wrapper checks dtype, dimensions, length and device before passing a bare
    pointer: a float32 h would be read past its end and its outputs overrun."""
    torch = pytest.importorskip("torch")
    f64, f32, i64 = torch.float64, torch.float32, torch.int64
    n = 8
    with pytest.raises(TypeError):
        B.check_tensor([1.0], "x", f64)
    with pytest.raises(TypeError):
        B.check_tensor(torch.zeros(n, dtype=f32), "x", f64)
    with pytest.raises(ValueError, match="dimension"):
        B.check_tensor(torch.zeros(2, n, dtype=f64), "x", f64, ndim=1)
    with pytest.raises(ValueError, match="shape"):
        B.check_tensor(torch.zeros(n + 1, dtype=f64), "x", f64, (n,))
    with pytest.raises(ValueError, match="CUDA"):
        B.check_tensor(torch.zeros(n, dtype=f64), "x", f64, (n,))  # a CPU tensor

    s = B.Solver.__new__(B.Solver)  # no context: every check must fire before the library
    s._torch, s.ctx, s.device, s.n = torch, None, 0, n
    cases = [
        (lambda: s.sort(torch.zeros(3, n, dtype=f32), torch.ones(n, dtype=f64)), TypeError),
        (lambda: s.sort(torch.zeros(n, 3, dtype=f64), torch.ones(n, dtype=f64)), ValueError),
        (lambda: s.sort(torch.zeros(3, n, dtype=f64), torch.ones(n, 1, dtype=f64)), ValueError),
        (lambda: s.sort(torch.zeros(3, n, dtype=f64), torch.ones(n, dtype=f64)), ValueError),  # CPU
        (lambda: s.solve(torch.ones(n, dtype=f32)), TypeError),
        (lambda: s.solve(torch.ones(n - 1, dtype=f64)), ValueError),
        (lambda: s.evaluate(torch.ones(n, dtype=f32)), TypeError),
        (lambda: s.evaluate(torch.ones(n + 1, dtype=f64)), ValueError),
        (lambda: s.knn(4, torch.ones(n, dtype=f32)), TypeError),
        (lambda: s.knn(4, torch.ones(2, n, dtype=f64)), ValueError),
        (lambda: s.autotune(torch.ones(n, dtype=f32)), TypeError),
        (lambda: s.interact(torch.ones(n, dtype=f64), torch.zeros(3, n, dtype=f32)), TypeError),
        (lambda: s.interact(torch.ones(n, dtype=f64), torch.zeros(n, 3, dtype=f64)), ValueError),
        (lambda: s.interact(torch.ones(n - 1, dtype=f64), torch.zeros(3, n, dtype=f64)), ValueError),
        (lambda: s.batch_solve(torch.tensor([0, n], dtype=torch.int32), torch.zeros(3, n, dtype=f64),
                               torch.ones(n, dtype=f64), torch.ones(n, dtype=f64),
                               torch.ones(1, dtype=f64), torch.ones(1, dtype=f64)), TypeError),
        (lambda: s.batch_solve(torch.tensor([0, n], dtype=i64), torch.zeros(3, n, dtype=f64),
                               torch.ones(n, dtype=f64), torch.ones(n, dtype=f64),
                               torch.ones(2, dtype=f64), torch.ones(1, dtype=f64)), ValueError),
    ]
    for call, err in cases:
        with pytest.raises(err):
            call()
    out = {"h": torch.ones(n, dtype=f64), "rho": torch.ones(n, dtype=f64), "count": torch.ones(n, dtype=f64),
           "nw": torch.ones(n, dtype=f64)}
    with pytest.raises(TypeError, match="count"):  # counts are int32
        s.solve(torch.ones(n, dtype=f64), out=out)
