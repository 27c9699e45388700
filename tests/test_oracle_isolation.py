"""The oracle is test infrastructure: nothing on the product path may reach it.

Static checks on the sources (CPU only): the package and the C sources never
import, load or include anything of `oracle/`, and bench.py touches the
oracle only in its CPU baselines and its reference arm (the functions named
below), so that every GPU figure bench.py prints comes from the CUDA library
alone.  A regression (an oracle call slipped into a GPU leg or into the
configurations' checks) fails here before any GPU run.
"""
import ast
import glob
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2108_08769_gb300")

# bench.py functions allowed to run the oracle: the single-core and all-core
# CPU baselines and the reference arm
BENCH_ORACLE_FUNCTIONS = {"cpu_baseline_sample", "_oracle_worker", "cpu_baseline_all_cores", "run_reference"}


def _imports_oracle(node):
    if isinstance(node, ast.Import):
        return any(a.name == "oracle" or a.name.startswith("oracle.") for a in node.names)
    if isinstance(node, ast.ImportFrom):
        return (node.module or "").split(".")[0] == "oracle"
    return False


def test_package_python_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "*.py")):
        tree = ast.parse(open(path).read(), path)
        assert not any(_imports_oracle(n) for n in ast.walk(tree)), path


def test_cuda_sources_and_headers_never_name_the_oracle_files():
    srcs = glob.glob(os.path.join(PKG, "csrc", "*")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    assert srcs
    for path in srcs:
        text = open(path).read()
        assert "ac_oracle" not in text and "liborc" not in text and "orc_" not in text, path


def test_bench_runs_the_oracle_only_in_its_cpu_baselines_and_reference_arm():
    path = os.path.join(ROOT, "bench.py")
    tree = ast.parse(open(path).read(), path)
    # no module-level import of the oracle
    assert not any(_imports_oracle(n) for n in tree.body)
    found = set()
    for fn in ast.walk(tree):
        if not isinstance(fn, (ast.FunctionDef, ast.AsyncFunctionDef)):
            continue
        if any(_imports_oracle(n) for n in ast.walk(fn)):
            found.add(fn.name)
    # nested functions are walked twice (alone and inside their parent): the
    # allowed set must cover every function whose body imports the oracle
    assert found <= BENCH_ORACLE_FUNCTIONS, found - BENCH_ORACLE_FUNCTIONS
    assert {"cpu_baseline_sample", "run_reference"} <= found
