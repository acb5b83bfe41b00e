"""The ctypes binding describes the C ABI of include/nk.h exactly: every
structure has the header's size and field offsets, and every constant the
binding uses has the header's value.  A C program compiled with gcc against
the header prints its own view of the layouts; no GPU and no libnk.so are
needed."""
import ctypes
import json
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2112_10526_gb300 import nk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

STRUCTS = ["nk_rbm", "nk_ham", "nk_qgt", "nk_rbm_symm", "nk_crbm", "nk_tdvp_cfg", "nk_chains", "nk_sr_cfg", "nk_request", "nk_result", "nk_server_stats"]

CONSTANTS = {
    "NK_OK": nk.NK_OK, "NK_ERR_INVALID_ARG": nk.NK_ERR_INVALID_ARG, "NK_ERR_CUDA": nk.NK_ERR_CUDA,
    "NK_ERR_OOM": nk.NK_ERR_OOM, "NK_ERR_TIMEOUT": nk.NK_ERR_TIMEOUT,
    "NK_ERR_NOT_CONVERGED": nk.NK_ERR_NOT_CONVERGED, "NK_ERR_UNIMPLEMENTED": nk.NK_ERR_UNIMPLEMENTED,
    "NK_F64": nk.NK_F64, "NK_MIXED": nk.NK_MIXED,
    "NK_RULE_LOCAL": nk.NK_RULE_LOCAL, "NK_RULE_EXCHANGE": nk.NK_RULE_EXCHANGE,
    "NK_RULE_HAMILTONIAN": nk.NK_RULE_HAMILTONIAN,
    "NK_TFIM": nk.NK_TFIM, "NK_HEIS": nk.NK_HEIS,
    "NK_SOLVER_CHOLESKY": nk.NK_SOLVER_CHOLESKY, "NK_SOLVER_CHOLESKY_SAMPLESPACE": nk.NK_SOLVER_CHOLESKY_SAMPLESPACE,
    "NK_SOLVER_CG": nk.NK_SOLVER_CG, "NK_SOLVER_SVD": nk.NK_SOLVER_SVD,
    "NK_SOLVER_SVD_SAMPLESPACE": nk.NK_SOLVER_SVD_SAMPLESPACE, "NK_QGT_ONTHEFLY": nk.NK_QGT_ONTHEFLY, "NK_QGT_JACOBIAN": nk.NK_QGT_JACOBIAN,
    "NK_TDVP_EULER": nk.NK_TDVP_EULER, "NK_TDVP_HEUN": nk.NK_TDVP_HEUN,
    "NK_REQ_EXPECT": nk.NK_REQ_EXPECT, "NK_REQ_SR_STEP": nk.NK_REQ_SR_STEP,
    "NK_PROF_SWEEP": nk.PROF_CLASSES["sweep"], "NK_PROF_ELOC": nk.PROF_CLASSES["eloc"],
    "NK_PROF_GRAM": nk.PROF_CLASSES["gram"], "NK_PROF_CHOL_UPDATE": nk.PROF_CLASSES["chol_update"],
    "NK_PROF_CHOL_PANEL": nk.PROF_CLASSES["chol_panel"], "NK_PROF_TRSV": nk.PROF_CLASSES["trsv"],
    "NK_PROF_JVP_VJP": nk.PROF_CLASSES["jvp_vjp"],
}


def _c_program():
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "nk.h"', "int main(void) {", 'printf("{");']
    for name in STRUCTS:
        cls = getattr(nk, name)
        lines.append(f'printf("\\"{name}\\": {{\\"size\\": %zu, \\"fields\\": {{", sizeof({name}));')
        for k, (field, _t) in enumerate(cls._fields_):
            sep = "," if k else ""
            lines.append(f'printf("{sep}\\"{field}\\": %zu", offsetof({name}, {field}));')
        lines.append('printf("}}, ");')
    lines.append('printf("\\"nk_sr_stats\\": {\\"size\\": %zu, \\"fields\\": {", sizeof(nk_sr_stats));')
    for k, field in enumerate(nk.SR_STATS_FIELDS):
        sep = "," if k else ""
        lines.append(f'printf("{sep}\\"{field}\\": %zu", offsetof(nk_sr_stats, {field}));')
    lines.append('printf("}}, \\"constants\\": {");')
    for k, c in enumerate(CONSTANTS):
        sep = "," if k else ""
        lines.append(f'printf("{sep}\\"{c}\\": %lld", (long long)({c}));')
    lines.append('printf("}}\\n"); return 0; }')
    return "\n".join(lines)


@pytest.fixture(scope="module")
def header_view():
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write(_c_program())
        subprocess.run(["gcc", "-std=c11", "-Wall", "-I", INCLUDE, src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


@pytest.mark.parametrize("name", STRUCTS)
def test_struct_layout_matches_header(header_view, name):
    cls = getattr(nk, name)
    view = header_view[name]
    assert ctypes.sizeof(cls) == view["size"], name
    for field, _t in cls._fields_:
        assert getattr(cls, field).offset == view["fields"][field], (name, field)


def test_sr_stats_is_a_row_of_doubles(header_view):
    view = header_view["nk_sr_stats"]
    assert view["size"] == 8 * nk.SR_STATS_DOUBLES
    for k, field in enumerate(nk.SR_STATS_FIELDS):
        assert view["fields"][field] == 8 * k, field


def test_constants_match_header(header_view):
    assert header_view["constants"] == CONSTANTS
