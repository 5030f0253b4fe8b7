"""The C ABI library loads and exports every function include/cva.h declares
(no GPU needed: nothing is called that touches a device)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cva.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cva_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("cva_model_create", "cva_fit", "cva_project", "cva_to_u8", "cva_project_u8", "cva_strerror"):
        assert n in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    import paper_1612_06457_gb300 as cva

    path = cva.build()
    lib = cva.load()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (cva_[a-z0-9_]+)", out))
    declared = set(_declared())
    assert declared <= exported, declared - exported
    for n in declared:
        getattr(lib, n)
        assert n in cva.SIGNATURES, n
    assert cva.cva_strerror(cva.CVA_ERR_NOT_SPD).startswith("within-class")


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA path are independent: neither includes or
    imports the other."""
    pkg = os.path.join(ROOT, "paper_1612_06457_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"(?:import|include)\s+\S*oracle\S*", text), f
                assert "cva_oracle" not in text, f
    osrc = open(os.path.join(ROOT, "oracle", "cva_oracle.c")).read()
    assert "cva.h" not in osrc and "csrc" not in osrc
