"""The C-ABI library loads and exports every entry point include/nis.h declares (no GPU
needed; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2401_14051_gb300", "libnis.so")


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^(?:nis_status|void|const char \*|size_t)\s*\*?\s*(nis_\w+)\(",
                                src, re.M)
    return names


@pytest.fixture(scope="module")
def built_lib():
    if not os.path.exists(LIB):
        from paper_2401_14051_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_every_declared_symbol_is_exported(built_lib):
    names = _declared()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(built_lib):
    from paper_2401_14051_gb300 import nis
    assert set(_declared()) <= set(nis._SIGS)


def test_create_without_gpu_reports_cuda_error(built_lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2401_14051_gb300 import nis
    with pytest.raises(nis.NisError) as e:
        nis.Context(0, torch_allocator=False)
    assert e.value.status == -5


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2401_14051_gb300 import nis
    monkeypatch.setattr(nis, "_lib", None)
    monkeypatch.setattr(nis, "LIB_PATH", str(tmp_path / "libnis.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        nis.lib()


def _imports(path):
    import ast
    tree = ast.parse(open(path).read())
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            out.add(node.module.split(".")[0])
    return out


def test_oracle_and_cuda_path_share_nothing():
    # the product package and the input generators never import the oracle, the oracle
    # never imports the product package, and no CUDA or C source reaches into oracle/
    pkg = os.path.join(ROOT, "paper_2401_14051_gb300")
    for base, names in ((pkg, ("oracle",)), (os.path.join(ROOT, "synth"), ("oracle", "paper_2401_14051_gb300"))):
        for dirpath, _, files in os.walk(base):
            for f in files:
                p = os.path.join(dirpath, f)
                if f.endswith(".py"):
                    assert not (_imports(p) & set(names)), p
                elif f.endswith((".cu", ".h", ".c", ".cpp")):
                    assert "oracle" not in open(p).read(), p
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            assert "paper_2401_14051_gb300" not in _imports(os.path.join(ROOT, "oracle", f))
    # outside tests/, only the smoke entry point and bench.py's CPU legs import the oracle
    users = {f for f in os.listdir(ROOT) if f.endswith(".py") and "oracle" in _imports(os.path.join(ROOT, f))}
    assert users <= {"__graft_entry__.py", "bench.py"}, users
