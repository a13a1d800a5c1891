"""The ctypes mirrors of the C-ABI structs and signatures (paper_1512_08401_gb300/wdb.py) against the header
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


def header_declarations() -> dict:
    """{function: (return type, [parameter types])} from include/wdb.h, comments stripped."""
    import re
    txt = open(os.path.join(ROOT, "include", "wdb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    txt = re.sub(r"//[^\n]*", "", txt)
    out = {}
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(wdb_\w+)\s*\(([^;{]*?)\)\s*;", txt):
        ret, name, params = " ".join(m.group(1).split()), m.group(2), " ".join(m.group(3).split())
        if ret.startswith("typedef") or "}" in ret:
            continue
        types = []
        if params not in ("", "void"):
            for p in params.split(","):
                p = p.strip()
                # drop the parameter name (the last identifier when more than a type is present)
                pm = re.match(r"^(.*?[\s\*])([A-Za-z_]\w*)$", p)
                types.append(" ".join((pm.group(1) if pm else p).replace("*", " * ").split()))
        out[name] = (" ".join(ret.replace("*", " * ").split()), types)
    return out


def ctype_for(c_type: str):
    """The ctypes type the binding must declare for a C type of the header."""
    t = c_type.replace("const ", "").strip()
    stars = t.count("*")
    base = t.replace("*", "").strip()
    mirrors = {name: cls for name, (cls, _) in STRUCTS.items()}
    if stars == 0:
        return {"int": ctypes.c_int, "wdb_status": ctypes.c_int, "long long": ctypes.c_longlong,
                "double": ctypes.c_double, "unsigned long long": ctypes.c_ulonglong, "void": None}[base]
    if stars == 1:
        if base == "double":
            return ctypes.POINTER(ctypes.c_double)
        if base == "int":
            return ctypes.POINTER(ctypes.c_int)
        if base == "float":
            return ("float*",)       # a device pointer (void*) or a host float array
        if base == "char":
            return ctypes.c_char_p
        if base in mirrors:
            return ctypes.POINTER(mirrors[base])
        return ctypes.c_void_p      # handles, streams, device pointers
    return ("pointer to pointer",)


def test_binding_signatures_match_header():
    decl = header_declarations()
    bound = wdb._SIGS
    assert set(bound) - set(decl) == set(), "bound but not declared"
    bad = []
    for name, (res, args) in bound.items():
        c_ret, c_args = decl[name]
        if len(args) != len(c_args):
            bad.append((name, "arity", len(args), len(c_args)))
            continue
        want_ret = ctype_for(c_ret)
        if c_ret.replace("const ", "").strip() == "const char *" or c_ret.endswith("char *"):
            want_ret = ctypes.c_char_p
        if want_ret is not res:
            bad.append((name, "return", res, c_ret))
        for k, (a, c) in enumerate(zip(args, c_args)):
            want = ctype_for(c)
            if want == ("float*",):
                ok = a in (ctypes.c_void_p, ctypes.POINTER(ctypes.c_float))
            elif want == ("pointer to pointer",):
                ok = a in (ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p)
            else:
                ok = a is want
            if not ok:
                bad.append((name, k, a, c))
    assert not bad, bad
