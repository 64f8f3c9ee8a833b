"""The C ABI library builds, loads and exports every symbol of include/eda.h
(no compute calls: these run without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "eda.h")).read()
    return sorted(set(re.findall(r"EDA_API\s+[\w\s\*]+?\b(eda_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["eda_create", "eda_destroy", "eda_set_trajectory", "eda_sketch", "eda_build_lmp",
              "eda_solve_batch", "eda_hvp", "eda_last_error"]:
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    import paper_2605_23571_gb300 as P
    P.build()
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(eda_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    assert set(P.EXPORTS) == set(declared_symbols())


def test_library_loads_and_binds():
    import paper_2605_23571_gb300 as P
    L = P.lib()
    for s in P.EXPORTS:
        assert hasattr(L, s)
    assert b"sm_103a" in L.eda_version()


def test_oracle_and_cuda_path_share_no_code():
    # neither side imports the other; only eda_synth is common
    pkg = os.path.join(ROOT, "paper_2605_23571_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"^\s*(?:import|from)\s+(\w+)", txt, re.M), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            imports = re.findall(r"^\s*(?:import|from)\s+([\w\.]+)", txt, re.M)
            assert not any(m.startswith("paper_2605_23571_gb300") for m in imports), f
