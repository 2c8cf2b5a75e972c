"""The C-ABI library builds, loads without a GPU and exports every symbol include/mrq.h declares."""
import ctypes
import os
import re

import paper_1909_06935_gb300 as P
from paper_1909_06935_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mrq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mrq_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("mrq_create", "mrq_destroy", "mrq_load_hamiltonian", "mrq_load_reference", "mrq_sample",
                     "mrq_debug_local", "mrq_finalize", "mrq_walkers_advance"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_header_sizes():
    # mrq_neighbour: 4 words + 5 doubles + 2 uint32 = 80 bytes; mrq_local: 6 doubles + 7 int64 = 104
    assert ctypes.sizeof(P.Neighbour) == 80
    assert ctypes.sizeof(P.Local) == 104
    assert ctypes.sizeof(P.SampleParams) == 64


def test_label_count_matches_generator():
    import synthetic as S
    for nc, nv in [(0, 0), (2, 6), (6, 40), (10, 80)]:
        assert P.n_labels(nc, nv) == S.n_labels(nc, nv)


def test_ctypes_layouts_match_the_c_header(tmp_path):
    """Compile a C program against include/mrq.h and compare struct sizes with the binding's."""
    import subprocess
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "mrq.h"\nint main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                   ' sizeof(mrq_sample_params), sizeof(mrq_result), sizeof(mrq_local), sizeof(mrq_neighbour),'
                   ' sizeof(mrq_server_params), sizeof(mrq_request), sizeof(mrq_request_status),'
                   ' sizeof(mrq_tune_result), sizeof(mrq_sci_params), sizeof(mrq_sci_result)); return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(t) for t in (P.SampleParams, P.Result, P.Local, P.Neighbour, P.ServerParams, P.Request,
                                       P.RequestStatus, P.TuneResult, P.SciParams, P.SciResult)]
    assert got == want
