"""CPU checks of the boundary: the library builds, loads, exports every entry
point that include/rrs.h declares, and reports errors without a GPU."""
import os
import re

import pytest

import paper_2506_08262_gb300 as rrs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rrs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:rrs_status|const char\*|uint64_t)\s+(rrs_\w+)\s*\(", text, flags=re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2506_08262_gb300 import build
    build.build()
    lib = rrs.load()
    decl = declared_functions()
    assert len(decl) >= 10
    for name in decl:
        assert hasattr(lib, name), name
    assert set(decl) == set(rrs.exported_symbols())


def test_status_strings_and_no_gpu_error():
    assert rrs.rrs_status_string(rrs.RRS_ERR_BUDGET) == "device memory budget exceeded"
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(rrs.RRSError) as e:
        rrs.rrs_create(0)
    assert e.value.status in (rrs.RRS_ERR_CUDA, rrs.RRS_ERR_INVALID_ARG)


def test_binding_constants_match_the_header():
    # the binding restates the header's numeric constants; a drift would silently misread profiler slots,
    # statuses or request fields
    text = open(os.path.join(ROOT, "include", "rrs.h")).read()
    defines = {k: int(v) for k, v in re.findall(r"#define\s+(RRS_\w+)\s+\(?(-?\d+)u?\)?", text)}
    stages = sorted((v, k) for k, v in defines.items() if k.startswith("RRS_STAGE_"))
    assert [v for v, _ in stages] == list(range(defines["RRS_NSTAGES"]))
    assert len(rrs.RRS_STAGES) == defines["RRS_NSTAGES"]
    for v, k in stages:
        assert rrs.RRS_STAGES[v] == k[len("RRS_STAGE_"):].lower(), (k, rrs.RRS_STAGES[v])
    for k, v in defines.items():
        if k.startswith(("RRS_ERR_", "RRS_PREC_", "RRS_F32", "RRS_F64", "RRS_HALFSPACE", "RRS_PROJECTION",
                         "RRS_ASYM_PROJECTION")) and hasattr(rrs, k):
            assert getattr(rrs, k) == v, k


def test_the_product_path_and_the_oracle_stay_apart():
    # the oracle is test infrastructure: the CUDA library and its binding never reference it, the oracle never
    # references the library, and bench.py touches it only in its CPU-baseline and reference-arm functions
    import ast

    pkg = os.path.join(ROOT, "paper_2506_08262_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b", text), os.path.join(dirpath, f)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            code = re.sub(r'""".*?"""|/\*.*?\*/|#[^\n]*', "", text, flags=re.S)
            assert "paper_2506_08262_gb300" not in code and "csrc" not in code and "rrs_device" not in code, f
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, (ast.Import, ast.ImportFrom)):
                    names = [a.name for a in node.names] + ([node.module] if isinstance(node, ast.ImportFrom) else [])
                    if any(n and n.split(".")[0] == "oracle" for n in names):
                        users.add(fn.name)
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert not any(a.name.split(".")[0] == "oracle" for n in top for a in n.names)
    assert users == {"oracle_sample_rate", "run_reference"}, users
