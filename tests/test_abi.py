"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, exports
every entry point declared in include/ephb.h, the ctypes structs match the C layout, and
the CUDA path and the oracle share no code."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2109_08547_gb300 import binding as B
from paper_2109_08547_gb300 import build as BU

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ephb.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:ephb_status|void|int64_t|int|const char \*)\s*(ephb_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_five_calls():
    names = _declared()
    for n in ("ephb_set_wannier_model", "ephb_build_meshes_ibz", "ephb_compute_transition_rates",
              "ephb_solve_coupled_bte", "ephb_transport_coefficients"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(BU.build())
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(_declared()) == set(B.EXPORTED)


def test_struct_layouts_match_header(tmp_path):
    structs = {"ephb_model": B.ModelC, "ephb_mesh_opts": B.MeshOptsC, "ephb_mesh_info": B.MeshInfoC,
               "ephb_thermo": B.ThermoC, "ephb_delta": B.DeltaC, "ephb_rates_info": B.RatesInfoC,
               "ephb_solve_opts": B.SolveOptsC, "ephb_solve_info": B.SolveInfoC, "ephb_coeffs": B.CoeffsC,
               "ephb_coeff_inputs": B.CoeffInputsC, "ephb_impurities": B.ImpuritiesC}
    src = tmp_path / "sz.c"
    lines = ['#include <stdio.h>', '#include "ephb.h"', "int main(void){"]
    for n in structs:
        lines.append(f'printf("%zu\\n", sizeof({n}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    sizes = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    for (n, cls), sz in zip(structs.items(), sizes):
        assert ctypes.sizeof(cls) == sz, n


def test_binding_constants_match_header():
    text = open(HEADER).read()
    for name, value in (("EPHB_MAX_ACCEL_DEPTH", B.MAX_ACCEL_DEPTH), ("EPHB_NFEAT", B.NFEAT),
                        ("EPHB_TUNE_TC_COLS", B.TUNE_TC_COLS), ("EPHB_TUNE_WITHHOLD_MMA", B.TUNE_WITHHOLD_MMA),
                        ("EPHB_NOALLOC_MAX_ITEMS", B.NOALLOC_MAX_ITEMS),
                        ("EPHB_TUNE_DEFER_INSTANCES", B.TUNE_DEFER_INSTANCES), ("EPHB_DELTA_TETRA", B.DELTA_TETRA),
                        ("EPHB_TUNE_STAGE_A_TMEM_A", B.TUNE_STAGE_A_TMEM_A), ("EPHB_MAX_DOPANTS", B.MAX_DOPANTS)):
        m = re.search(r"#define\s+%s\s+(\d+)" % name, text)
        assert m and int(m.group(1)) == value, name


def test_create_without_device_fails_cleanly():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is visible")
    except ImportError:
        pass
    lib = B.load()
    h = ctypes.c_void_p()
    st = lib.ephb_create(ctypes.byref(h), 0, None)
    assert st == B.ECUDA and not h.value
    assert lib.ephb_last_error(None) == b"null context"
    assert lib.ephb_set_wannier_model(None, None) == B.EINVAL


def test_cuda_path_and_oracle_share_no_code():
    pkg = os.path.join(ROOT, "paper_2109_08547_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f
                assert "oracle/" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "binding" not in txt and "csrc" not in txt and "libephb" not in txt, f
            for m in re.findall(r"^\s*(?:from|import)\s+([\w.]+)", txt, re.M):
                assert m.split(".")[0] in ("numpy", "dataclasses", "__future__") or m.startswith("."), m
