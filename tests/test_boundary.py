"""The boundary between the product path, the oracle and the input generators.

* The package (Python binding, engine, warm-start wrapper, build script) and its native sources
  never import, include or name a file of the oracle, and the oracle never imports the package:
  parity compares two implementations that share no code.
* The seeded input generators import neither side.
* With the shared library absent the binding raises instead of falling back to anything, and the
  torch-facing engine rejects host tensors before it reaches the library: there is no CPU path.
All checks read the sources (AST imports, preprocessor includes) or run on the host.
"""
import ast
import pathlib

import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]
PKG = ROOT / "paper_2406_06640_gb300"


def _imports(path: pathlib.Path):
    """Top-level module names imported by one Python file (absolute imports; relative ones as '.')."""
    tree = ast.parse(path.read_text(), filename=str(path))
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            names.add("." if node.level else node.module.split(".")[0])
    return names


def _py_files(d: pathlib.Path):
    return sorted(p for p in d.rglob("*.py") if "_build" not in p.parts and "__pycache__" not in p.parts)


def test_package_never_imports_the_oracle_or_the_generators():
    files = _py_files(PKG)
    assert files, "package sources not found"
    for f in files:
        bad = _imports(f) & {"oracle", "synth", "tests"}
        assert not bad, f"{f.relative_to(ROOT)} imports {sorted(bad)}"


def test_native_sources_include_nothing_from_the_oracle():
    srcs = sorted(list((PKG / "csrc").rglob("*.cu")) + list((PKG / "csrc").rglob("*.cuh")) +
                  list((PKG / "csrc").rglob("*.h")) + list((ROOT / "include").rglob("*.h")))
    assert srcs, "native sources not found"
    for f in srcs:
        for line in f.read_text().splitlines():
            s = line.strip()
            if s.startswith("#include"):
                assert "oracle" not in s and "synth" not in s, f"{f.relative_to(ROOT)}: {s}"


def test_oracle_never_imports_the_package():
    files = _py_files(ROOT / "oracle")
    assert files
    for f in files:
        bad = _imports(f) & {PKG.name, "synth", "torch", "ctypes"}
        assert not bad, f"{f.relative_to(ROOT)} imports {sorted(bad)}"


def test_generators_import_neither_side():
    files = _py_files(ROOT / "synth")
    assert files
    for f in files:
        bad = _imports(f) & {PKG.name, "oracle", "torch", "ctypes"}
        assert not bad, f"{f.relative_to(ROOT)} imports {sorted(bad)}"


def test_missing_library_raises_instead_of_falling_back(monkeypatch, tmp_path):
    from paper_2406_06640_gb300 import binding
    from paper_2406_06640_gb300 import build as _build

    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "absent" / "libptycho.so"))
    monkeypatch.setattr(_build, "up_to_date", lambda: True)
    with pytest.raises(ImportError, match="libptycho.so not found"):
        binding.load(build_if_missing=False)
    with pytest.raises(ImportError):
        binding.load()
    # every entry point goes through load(): a plan cannot be made without the library
    with pytest.raises(ImportError):
        binding.Plan({"M": 8, "K": 1, "N": 1}, 0, 0)


def test_engine_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    from paper_2406_06640_gb300 import engine

    I = torch.zeros(2, 8, 8, dtype=torch.float32)
    pos = torch.zeros(2, 2, dtype=torch.int32)
    with pytest.raises(ValueError, match="CUDA tensor"):
        engine.Reconstruction({"M": 8, "K": 1, "N": 2}, I, pos)
