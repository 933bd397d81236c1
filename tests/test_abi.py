"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/sky.h declares (no compute calls: CPU only)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sky.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sky_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1610_07522_gb300 import build
    return build.build()


def test_header_declares_the_hot_path():
    names = set(_declared())
    for n in ("sky_init", "sky_apply_h", "sky_damped_step", "sky_overlap", "sky_orthonormalize",
              "sky_subspace_diag", "sky_rotate", "sky_densities", "sky_mean_fields", "sky_energy"):
        assert n in names


def test_header_is_plain_c(tmp_path):
    """The boundary is a C ABI: the header compiles as strict C99 on its own."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "uses_sky.c"
    src.write_text('#include "sky.h"\nint main(void) { return sky_supported_size(16, SKY_F64) != 1; }\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o",
                        str(tmp_path / "uses_sky.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(sky_[a-z_0-9]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binds(libpath):
    L = ctypes.CDLL(libpath)
    for n in _declared():
        assert hasattr(L, n)
    from paper_1610_07522_gb300 import binding
    assert binding.lib() is not None
    assert binding.sky_supported_size(24, binding.SKY_F64)
    assert not binding.sky_supported_size(64, binding.SKY_F64)
    assert binding.sky_supported_size(64, binding.SKY_F32)
    assert not binding.sky_supported_size(7, binding.SKY_F32)


def test_binding_marshals_struct_layout():
    from paper_1610_07522_gb300 import binding
    from paper_1610_07522_gb300 import inputs as IN
    s = binding.skyrme_struct(IN.SLY4, True)
    assert ctypes.sizeof(s) == 13 * 8 + 8   # 13 doubles + int padded
    assert s.t3 == IN.SLY4["t3"] and s.coulomb == 1


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle (it is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_1610_07522_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_binding_net_constants_match_header():
    from paper_1610_07522_gb300 import binding
    from oracle import precond_oracle as P
    src = open(os.path.join(ROOT, "include", "sky.h")).read()
    defs = dict(re.findall(r"#define\s+(SKY_NET_[A-Z_]+)\s+([0-9.]+)", src))
    assert len(defs) == 6
    for k, v in defs.items():
        assert float(getattr(binding, k)) == float(v), k
    assert binding.SKY_NET_NPARAM == P.NPARAM
    assert binding.SKY_NET_WMAX == P.WMAX and binding.SKY_NET_HIDDEN == P.HIDDEN
    assert binding.SKY_NET_USCALE == P.U_SCALE and binding.SKY_NET_WSCALE == P.W_SCALE


def test_binding_eigen_knob_matches_header():
    from paper_1610_07522_gb300 import binding
    src = open(os.path.join(ROOT, "include", "sky.h")).read()
    assert re.search(r"SKY_KNOB_EIGEN_METHOD\s*=\s*(\d+)", src).group(1) == str(binding.SKY_KNOB_EIGEN_METHOD)
    enum = re.search(r"enum\s*\{\s*SKY_EIG_AUTO\s*=\s*(\d+),\s*SKY_EIG_JACOBI\s*=\s*(\d+),\s*"
                     r"SKY_EIG_TRIDIAGONAL\s*=\s*(\d+)\s*\}", src)
    assert tuple(int(x) for x in enum.groups()) == (binding.SKY_EIG_AUTO, binding.SKY_EIG_JACOBI,
                                                     binding.SKY_EIG_TRIDIAGONAL)


def test_binding_knobs_match_header():
    """Every tunable knob the header enumerates has the same value in the
    binding (the knobs travel as plain ints across the C ABI)."""
    from paper_1610_07522_gb300 import binding
    src = open(os.path.join(ROOT, "include", "sky.h")).read()
    body = re.search(r"typedef enum \{([^}]*)\} sky_knob;", src).group(1)
    knobs = dict((k, int(v)) for k, v in re.findall(r"(SKY_KNOB_[A-Z0-9_]+)\s*=\s*(\d+)", body))
    assert len(knobs) >= 13
    for k, v in knobs.items():
        assert getattr(binding, k) == v, k


def test_solver_eigen_method_sets_every_context(monkeypatch):
    """Solver.set_eigen_method and bench.py --eigen set the knob once on each
    distinct context (host logic only: the contexts are stand-ins)."""
    from paper_1610_07522_gb300 import binding
    from paper_1610_07522_gb300.solver import Solver
    import bench
    calls = []
    monkeypatch.setattr(binding, "sky_tune_set", lambda c, k, v: calls.append((c, k, v)))
    s = object.__new__(Solver)
    a, b = object(), object()
    for ctxq, want in (([a, a], [a]), ([a, b], [a, b])):
        calls.clear()
        s.ctxq = ctxq
        s.set_eigen_method(bench.EIGEN["jacobi"])
        assert [c for c, _, _ in calls] == want
        assert all(k == binding.SKY_KNOB_EIGEN_METHOD and v == binding.SKY_EIG_JACOBI for _, k, v in calls)
    assert bench.EIGEN == {"auto": binding.SKY_EIG_AUTO, "jacobi": binding.SKY_EIG_JACOBI,
                           "tridiagonal": binding.SKY_EIG_TRIDIAGONAL}
