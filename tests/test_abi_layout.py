"""The ctypes mirrors of the C-ABI structs (paper_1512_08401_gb300/wdb.py) against the header
(include/wdb.h): a small C program compiled against the header prints each struct's size and
the offset of every field, in declaration order, and both must equal the ctypes layout. A field
added to one side only, reordered or given another type fails here (no GPU needed)."""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1512_08401_gb300 import wdb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C field names in declaration order (typed from the header, not derived from the binding)
STRUCTS = {
    "wdb_theta_info": (wdb.ThetaInfo, ["n_rows", "n_cols", "levels", "n_subbands", "wavelet_taps", "rule",
                                       "K_requested", "K_eff", "n_taps", "n_candidates", "theta_max_abs",
                                       "phase_table_len", "build_ms", "plan_tuned", "plan_items",
                                       "plan_split_tiles", "plan_super_subbands", "plan_groups",
                                       "plan_smem_bytes", "plan_grid"]),
    "wdb_solve_params": (wdb.SolveParams, ["lambda", "w_subband_host", "max_iters", "tol", "precond",
                                           "jacobi_eps", "check_every", "x_init_dev", "no_graph",
                                           "target_objective", "time_kernels", "kkt_check", "ista", "fused",
                                           "spin_limit"]),
    "wdb_solve_result": (wdb.SolveResult, ["iters", "objective", "primal", "gap", "rel_gap", "support", "tau",
                                           "L_hat", "solve_ms", "ms_k1", "ms_k2", "timed_chunks",
                                           "first_primal_below", "status", "kkt_off", "kkt_on", "gap64",
                                           "rel_gap64"]),
    "wdb_kkt_result": (wdb.KktResult, ["objective", "gap", "rel_gap", "kkt_off", "kkt_on", "gmax", "support"]),
    "wdb_plan_summary": (wdb.PlanSummary, ["items", "pairs", "batches", "split_tiles", "super_subbands",
                                           "smem_bytes", "macs", "groups"]),
    "wdb_vtheta_info": (wdb.VThetaInfo, ["n_rows", "n_cols", "levels", "n_subbands", "rule", "K_requested",
                                         "K_eff", "n_taps", "n_candidates", "candidate_slots", "n_probes",
                                         "n_classes", "n_plan_rows", "plan_taps", "theta_max_abs", "build_ms"]),
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "wdb.h"', "int main(void) {"]
    for name, (_, fields) in STRUCTS.items():
        args = ", ".join(f"offsetof({name}, {f})" for f in fields)
        fmt = " ".join(["%zu"] * (len(fields) + 1))
        lines.append(f'    printf("{name} {fmt}\\n", sizeof({name}), {args});')
    lines += ["    return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {ln.split()[0]: [int(v) for v in ln.split()[1:]] for ln in out.splitlines()}


@pytest.mark.parametrize("name", sorted(STRUCTS))
def test_ctypes_struct_matches_header(c_layout, name):
    cls, fields = STRUCTS[name]
    got = c_layout[name]
    assert len(cls._fields_) == len(fields), (name, [f for f, _ in cls._fields_], fields)
    assert ctypes.sizeof(cls) == got[0], (name, ctypes.sizeof(cls), got[0])
    py_offsets = [getattr(cls, f).offset for f, _ in cls._fields_]
    assert py_offsets == got[1:], (name, list(zip(fields, got[1:], py_offsets)))
