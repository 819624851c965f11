"""The C ABI library loads and exports every entry point declared in
include/ds.h and include/ds_serve.h; the Python binding's structs match the header's layout
(compiled with gcc).  No GPU needed: nothing here launches work."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2503_13092_b300 import build as ds_build
from paper_2503_13092_b300 import ds

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("ds.h", "ds_serve.h")]


@pytest.fixture(scope="module")
def libpath():
    return ds_build.build()


def declared_symbols():
    txt = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"^DS_API [^(]*?\b(ds_\w+)\(", txt, re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("ds_load_geometry", "ds_load_nn_weights", "ds_reconstruct", "ds_vertex"):
        assert n in names
    assert sorted(ds.EXPORTED) == names          # the binding wraps every declared call


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (ds_\w+)$", out, re.M))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)            # loads without a GPU
    for n in declared_symbols():
        assert hasattr(lib, n)


def test_struct_layout_matches_header(tmp_path):
    structs = {"ds_geometry": ds.ds_geometry, "ds_nn_weights": ds.ds_nn_weights, "ds_params": ds.ds_params,
               "ds_event_batch": ds.ds_event_batch, "ds_seeds": ds.ds_seeds, "ds_ut_hits": ds.ds_ut_hits,
               "ds_tracks": ds.ds_tracks, "ds_vertices": ds.ds_vertices, "ds_stats": ds.ds_stats,
               "ds_kernel_time": ds.ds_kernel_time, "ds_tuning": ds.ds_tuning, "ds_tune_entry": ds.ds_tune_entry,
               "ds_server_config": ds.ds_server_config, "ds_request": ds.ds_request,
               "ds_completion": ds.ds_completion, "ds_server_stats": ds.ds_server_stats}
    dtypes = {"ds_track": ds.TRACK_DTYPE, "ds_vertex_rec": ds.VERTEX_DTYPE, "ds_vertex_info": ds.VINFO_DTYPE}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ds.h"', '#include "ds_serve.h"', 'int main(void){']
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    for name, dt in dtypes.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in dt.names:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).split("\n") if l)
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
    for name, dt in dtypes.items():
        assert int(got[name]) == dt.itemsize, name
        for f in dt.names:
            assert int(got[f"{name}.{f}"]) == dt.fields[f][1], (name, f)


def test_host_side_errors_without_gpu(libpath):
    """Calls that fail on the host return a status without touching a device."""
    L = ds.lib()
    assert L.ds_create(None, 0) == ds.DS_ERR_ARG
    p = ds.ds_default_params()
    assert p.k1 == 10 and p.nn_threshold == 0.5 and p.doca_max == 2.0
    assert ds.ds_status_string(ds.DS_ERR_CAPACITY) == "output capacity exceeded"
    h = ctypes.c_void_p()
    assert L.ds_create(ctypes.byref(h), 0) in (ds.DS_OK, ds.DS_ERR_CUDA)
    if h.value:
        L.ds_destroy(h)


def test_server_default_config(libpath):
    """The serving defaults (no device involved): four slots, graphs on, and
    inputs below 1 MiB per array gathered from pinned host memory."""
    c = ds.ds_server_default_config()
    assert (c.n_slots, c.graphs, c.gather_max_bytes) == (4, 1, 1 << 20)
    assert c.max_batch_events == 1024 and c.mlp_precision == ds.DS_MLP_FP32
