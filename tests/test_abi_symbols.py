"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/fiedler.h declares; the ctypes structs match the header's layout."""
import ctypes as C
import os
import re

import pytest

from paper_1602_04386_gb300 import build, fiedler

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fiedler.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fiedler.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fiedler_[a-z_]+)\s*\(", src)))


def test_header_declares_what_the_binding_lists():
    assert declared_functions() == sorted(fiedler.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_calls_that_need_no_gpu(lib):
    o = fiedler.fiedler_options_default()
    assert o.coarse_max_n == 25 and o.pi_cos_tol == 1e-6 and o.gs_sweeps == 2
    assert o.precision == fiedler.FIEDLER_FP32_FP64RED and o.max_levels == 30
    assert fiedler.fiedler_status_str(fiedler.FIEDLER_EDISCONNECTED) == "graph is not connected"
    assert fiedler.fiedler_plan_num_levels(None) == 0
    st, _ = fiedler.fiedler_plan_level_info(None, 0)
    assert st == fiedler.FIEDLER_EINVAL
    st, ids = fiedler.fiedler_poll_any(None, 4, 0)
    assert st == fiedler.FIEDLER_EINVAL and ids == []


def test_plan_fails_loudly_without_a_gpu(lib):
    """No CPU fallback: on a machine without a usable GPU, creating a plan
    reports a CUDA error and the binding raises."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fiedler.FiedlerError) as e:
        fiedler.Plan()
    assert e.value.status == fiedler.FIEDLER_ECUDA


def _offsets(struct):
    return [getattr(struct, f[0]).offset for f in struct._fields_]


def test_struct_layouts_match_header():
    # sizes computed by the C compiler from the header itself
    import subprocess
    import tempfile
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "fiedler.h"
int main(void){
 printf("%zu %zu %zu %zu %zu\n", sizeof(fiedler_options), sizeof(fiedler_graph), sizeof(fiedler_result),
        sizeof(fiedler_level_info), sizeof(fiedler_profile));
 printf("%zu %zu %zu %zu\n", offsetof(fiedler_options, seed), offsetof(fiedler_result, x),
        offsetof(fiedler_result, bad_index), offsetof(fiedler_profile, phase_bytes));
 printf("%zu\n", offsetof(fiedler_level_info, phase_ms));
 printf("%zu %zu %zu %zu\n", sizeof(fiedler_tuning), sizeof(fiedler_serving_stats),
        offsetof(fiedler_serving_stats, mean_blocks), offsetof(fiedler_options, batch_threads));
 return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    sizes = [int(v) for v in out[:5]]
    offs = [int(v) for v in out[5:9]]
    assert int(out[9]) == fiedler.fiedler_level_info.phase_ms.offset
    assert [int(v) for v in out[10:14]] == [C.sizeof(fiedler.fiedler_tuning), C.sizeof(fiedler.fiedler_serving_stats),
                                             fiedler.fiedler_serving_stats.mean_blocks.offset,
                                             fiedler.fiedler_options.batch_threads.offset]
    assert sizes == [C.sizeof(fiedler.fiedler_options), C.sizeof(fiedler.fiedler_graph),
                     C.sizeof(fiedler.fiedler_result), C.sizeof(fiedler.fiedler_level_info),
                     C.sizeof(fiedler.fiedler_profile)]
    assert offs == [fiedler.fiedler_options.seed.offset, fiedler.fiedler_result.x.offset,
                    fiedler.fiedler_result.bad_index.offset, fiedler.fiedler_profile.phase_bytes.offset]


def test_c_program_links_and_runs(lib):
    """A plain C program includes the header, links the library and calls the
    entry points that need no GPU; without a usable GPU, plan creation returns
    a CUDA error and a NULL plan."""
    import subprocess
    import tempfile
    import torch
    src = r'''
#include <stdio.h>
#include "fiedler.h"
int main(void) {
  fiedler_options o;
  fiedler_options_default(&o);
  if (o.coarse_max_n != 25) return 2;
  printf("%s\n", fiedler_status_str(FIEDLER_EDISCONNECTED));
  fiedler_plan *p = (fiedler_plan *)1;
  fiedler_status st = fiedler_plan_create(&o, NULL, &p);
  printf("%d %d\n", (int)st, p == NULL);
  if (st == FIEDLER_OK) fiedler_plan_destroy(p);
  return 0;
}
'''
    libdir = os.path.dirname(build.LIB)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe, "-L", libdir, "-lfiedler",
                               "-Wl,-rpath," + libdir])
        out = subprocess.check_output([exe], timeout=120).decode().split("\n")
    assert out[0] == "graph is not connected"
    st, null = (int(v) for v in out[1].split())
    if not torch.cuda.is_available():
        assert st == fiedler.FIEDLER_ECUDA and null == 1
