"""The product path has no CPU fallback and never reaches the oracle, checked on the CPU:
the binding refuses to import without its compiled library, no module of the package imports
the oracle, and the benchmark and entry module import it only in the legs allowed to (the
timed CPU baseline, the reference arm that times the oracle, the smoke check, and the build
step that compiles the checker)."""
import ast
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2212_14191_gb300")


def _oracle_imports(path):
    """(enclosing top-level function or None, line) of every import of the oracle package."""
    tree = ast.parse(open(path).read(), path)
    found = []

    def visit(node, owner):
        for child in ast.iter_child_nodes(node):
            o = owner
            if owner is None and isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)):
                o = child.name
            if isinstance(child, ast.Import):
                if any(a.name == "oracle" or a.name.startswith("oracle.") for a in child.names):
                    found.append((o, child.lineno))
            elif isinstance(child, ast.ImportFrom):
                if child.module and (child.module == "oracle" or child.module.startswith("oracle.")):
                    found.append((o, child.lineno))
            visit(child, o)

    visit(tree, None)
    return found


def test_package_never_imports_the_oracle():
    files = []
    for d, _, names in os.walk(PKG):
        files += [os.path.join(d, n) for n in names if n.endswith(".py")]
    assert len(files) >= 5
    for f in files:
        assert _oracle_imports(f) == [], f
    for d, _, names in os.walk(os.path.join(PKG, "csrc")):
        for n in names:
            src = open(os.path.join(d, n), errors="replace").read()
            assert "ntt_oracle" not in src and "oracle/" not in src, n


def test_oracle_is_imported_only_by_the_allowed_legs():
    bench = _oracle_imports(os.path.join(ROOT, "bench.py"))
    assert bench and {o for o, _ in bench} <= {"cpu_oracle_kops", "cpu_oracle_hmult", "reference_arm"}
    entry = _oracle_imports(os.path.join(ROOT, "__graft_entry__.py"))
    assert entry and {o for o, _ in entry} <= {"build", "smoke"}


def test_binding_refuses_to_import_without_the_library(tmp_path):
    pkg = tmp_path / "paper_2212_14191_gb300"
    pkg.mkdir()
    (pkg / "__init__.py").write_text("")
    shutil.copy(os.path.join(PKG, "fhe.py"), pkg / "fhe.py")
    r = subprocess.run([sys.executable, "-c", "from paper_2212_14191_gb300 import fhe"],
                       cwd=str(tmp_path), capture_output=True, text=True, timeout=120,
                       env={**os.environ, "PYTHONPATH": str(tmp_path)})
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "libfhe.so is not built" in r.stderr
