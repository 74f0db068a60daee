"""The C ABI library builds, loads and exports every entry point include/lorads.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

from oracle import Params
from paper_2403_09133_gb300 import lorads as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lorads.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lorads_[A-Za-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_mirrors_structs(lib):
    pb, rb, sb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib.lorads_struct_sizes(ctypes.byref(pb), ctypes.byref(rb), ctypes.byref(sb))
    assert pb.value == ctypes.sizeof(L.lorads_params)
    assert rb.value == ctypes.sizeof(L.lorads_result)
    assert sb.value == ctypes.sizeof(L.lorads_state)


def test_default_allocator_is_cuda_malloc(lib):
    # both callbacks NULL: the library's own cudaMalloc / cudaFree
    p = L.lorads_default_params()
    assert not p.dev_alloc and not p.dev_free and not p.alloc_ctx


def test_binding_exposes_same_names(lib):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_default_params_match_oracle_readings(lib):
    p = L.lorads_default_params()
    o = Params()
    assert p.tol == o.tol and p.rho_max == o.rho_max and p.rho_growth == o.rho_growth
    assert p.rho_every == o.rho_every and p.rank_factor == o.rank_factor
    assert p.cg_rel_tol == o.cg_rel_tol and p.cg_abs_floor == o.cg_abs_floor
    assert p.lbfgs_mem == o.lbfgs_mem and p.inner_max_iter == o.inner_max_iter
    assert p.inner_tol_factor == o.inner_tol_factor and p.inner_tol_max == o.inner_tol_max
    assert p.sigma_factor == o.sigma_factor and p.sigma_decrease == o.sigma_decrease
    assert p.sigma_max == o.sigma_max
    assert p.new_col_std == o.new_col_std
    assert p.max_admm_iter == o.max_admm_iter and p.max_outer == o.max_outer
    # "auto" resolves by problem class on both sides (library: < 0, oracle: None)
    assert p.gamma_scale < 0 and o.gamma_scale is None
    assert p.switch_tol < 0 and o.switch_tol is None and p.h < 0 and o.h is None
    assert p.kkt_dinf == int(o.kkt_dinf) and p.dinf_every == o.dinf_every
    assert p.escape_scale == o.escape_scale and p.lanczos_steps > 0
    assert p.subsolver == L.LORADS_SUB_CG and o.subsolver == "cg"
    assert p.polish == 1 and o.polish == "auto"
    assert p.newton_max == o.newton_max and p.newton_cg_max == o.newton_cg_max
    assert p.barrier_polls == 0          # library default: about a few seconds of polling
    assert p.lanczos_store_mb == 2048    # the dual tests' Lanczos blocks kept up to 2 GiB


def test_status_strings(lib):
    for code in range(0, -11, -1):
        assert L.lorads_status_string(code) != "unknown status"
    assert L.lorads_status_string(-99) == "unknown status"


def test_null_arguments_rejected(lib):
    assert lib.lorads_set_b(None, None) == L.LORADS_ERR_ARG
    assert lib.lorads_solve(None, None, None, None) == L.LORADS_ERR_ARG
    assert lib.lorads_create(0, 5, None) == L.LORADS_ERR_ARG


def test_field_offsets_match_header(tmp_path):
    """Every field of the binding's three structs sits where include/lorads.h puts it
    (offsetof from a C program compiled against the header), not only the sizes."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    structs = [("lorads_params", L.lorads_params), ("lorads_result", L.lorads_result),
               ("lorads_state", L.lorads_state)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lorads.h"',
             "int main(void) {"]
    for cname, py in structs:
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "offsets.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "offsets"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    for cname, py in structs:
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)
