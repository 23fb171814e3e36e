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
