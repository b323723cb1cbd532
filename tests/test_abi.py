"""C-ABI checks that need no GPU: libadg.so builds, loads and exports every
symbol include/adg.h declares; the ctypes structs match the C layouts; host
validation paths return error codes without touching a device."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "adg.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2007_03678_gb300 import adg, build
    build.build()
    return adg.load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(adg_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    from paper_2007_03678_gb300 import adg
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(adg.EXPORTS) == names


def test_struct_layouts_match_header():
    """Compile a probe against include/adg.h with the host compiler and
    compare sizeof/offsetof with the ctypes mirrors."""
    from paper_2007_03678_gb300 import adg
    probe = r"""
#include <stdio.h>
#include <stddef.h>
#include "adg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(adg_forcefield), sizeof(adg_grid_desc),
         sizeof(adg_ligand_desc), sizeof(adg_search_params), sizeof(adg_result), sizeof(adg_dock_trace),
         sizeof(adg_stats), sizeof(adg_ligand_stats), sizeof(adg_tuned_shape), sizeof(adg_peaks),
         sizeof(adg_schedule_stats));
  printf("%zu %zu %zu %zu %zu %zu\n", offsetof(adg_search_params, seed), offsetof(adg_search_params, mut_tors),
         offsetof(adg_result, genes), offsetof(adg_result, xyz), offsetof(adg_forcefield, k_out),
         offsetof(adg_peaks, gather_bytes));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(src, "w").write(probe)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    sizes = [int(x) for x in out[:11]]
    offs = [int(x) for x in out[11:]]
    assert sizes == [C.sizeof(adg.adg_forcefield), C.sizeof(adg.adg_grid_desc), C.sizeof(adg.adg_ligand_desc),
                     C.sizeof(adg.adg_search_params), C.sizeof(adg.adg_result), C.sizeof(adg.adg_dock_trace),
                     C.sizeof(adg.adg_stats), C.sizeof(adg.adg_ligand_stats), C.sizeof(adg.adg_tuned_shape),
                     C.sizeof(adg.adg_peaks), C.sizeof(adg.adg_schedule_stats)]
    assert offs == [adg.adg_search_params.seed.offset, adg.adg_search_params.mut_tors.offset,
                    adg.adg_result.genes.offset, adg.adg_result.xyz.offset, adg.adg_forcefield.k_out.offset,
                    adg.adg_peaks.gather_bytes.offset]


def test_strerror_and_defaults(lib):
    from paper_2007_03678_gb300 import adg
    assert lib.adg_strerror(0) == b"ok"
    for code in range(-8, 0):
        assert lib.adg_strerror(code) not in (b"", b"unknown error")
    assert lib.adg_strerror(-99) == b"unknown error"
    p = adg.search_params()
    assert (p.pop_size, p.nev, p.ls_method, p.ls_max_iters, p.elitism) == (150, 2500000, 1, 300, 1)
    assert p.crossover_rate == pytest.approx(0.8) and p.mutation_rate == pytest.approx(0.02)
    assert p.tournament_rate == pytest.approx(0.6) and p.seed == 42


def test_null_arguments_are_rejected(lib):
    from paper_2007_03678_gb300 import adg
    assert lib.adg_ctx_create(None, 0, None) == adg.ADG_OK - 1
    assert lib.adg_sync(None) == -1
    assert lib.adg_score(None, None, None, None, 0, None, None, 0) == -1
    assert lib.adg_ligand_info(None, None) == -1
    assert lib.adg_dock(None, None, None, 0, None, None, None) == -1
    assert lib.adg_receptor_destroy(None) == -1
    assert lib.adg_ligand_destroy(None) == -1
    assert lib.adg_ctx_set_geometry(None, 1) == -1
    assert lib.adg_ctx_tuned(None, None, 0, None) == -1
    assert lib.adg_probe_peaks(None, None) == -1
    assert lib.adg_score_multi(None, None, None, 0, None, None, None, None, 0) == -1


def test_no_gpu_context_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.adg_ctx_create(C.byref(h), 0, None) == -1
    assert not h.value


def test_product_package_does_not_reach_the_oracle():
    """The CUDA path's package neither imports nor names the oracle."""
    pkg = os.path.join(ROOT, "paper_2007_03678_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "adg_oracle" not in text and "orc_" not in text, f
