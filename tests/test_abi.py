"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/ml.h declares, and the ctypes mirrors of its structs have
the C layout."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import paper_2308_14278_gb300 as ml
from paper_2308_14278_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ml.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ml_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    return build.build_library()


def test_header_and_binding_agree():
    assert sorted(ml.EXPORTS) == declared_functions()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ml_[a-z0-9_]+)$", out, flags=re.M))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    lib = C.CDLL(libpath)
    for f in declared_functions():
        assert hasattr(lib, f)


def test_abi_version_and_error_string(libpath):
    lib = ml.load(libpath)
    assert lib.ml_abi_version() == ml.ABI_VERSION
    # a NULL descriptor is rejected before any CUDA call
    h = C.c_void_p()
    st = lib.ml_field_create(None, None, C.byref(h))
    assert st == 1 and h.value is None
    assert b"desc is NULL" in lib.ml_last_error()
    d = ml.FieldDesc()
    d.abi_version = 99
    assert lib.ml_field_create(C.byref(d), None, C.byref(h)) == 1
    assert b"abi_version" in lib.ml_last_error()
    assert lib.ml_field_destroy(None) == 0


@pytest.mark.parametrize("bad", [
    dict(map_nx=0), dict(map_x1=-2.0), dict(n_lens=5), dict(precision=7), dict(deposit=3),
    dict(taylor_p=17), dict(kappa_star=-1.0), dict(sheet_radius=-1.0), dict(l2_sub_x=-1), dict(l2_sub_y=5000),
])
def test_descriptor_validation_without_gpu(libpath, bad):
    lib = ml.load(libpath)
    d = ml.FieldDesc()
    d.abi_version = ml.ABI_VERSION
    d.map_x0, d.map_y0, d.map_x1, d.map_y1 = -1, -1, 1, 1
    d.map_nx = d.map_ny = 8
    d.n_av = 10
    for k, v in bad.items():
        setattr(d, k, v)
    h = C.c_void_p()
    assert lib.ml_field_create(C.byref(d), None, C.byref(h)) == 1   # ML_ERR_INVALID_ARG
    assert h.value is None


_LAYOUT_C = r"""
#include <stddef.h>
#include <stdio.h>
#include "ml.h"
#define P(T, f) printf(#T " " #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("ml_field_desc size %zu\n", sizeof(ml_field_desc));
  printf("ml_field_params size %zu\n", sizeof(ml_field_params));
  %FIELDS%
  return 0;
}
"""


def test_struct_layout_matches_header(tmp_path):
    lines = []
    for T, S in (("ml_field_desc", ml.FieldDesc), ("ml_field_params", ml.FieldParams)):
        for name, _ in S._fields_:
            lines.append(f"P({T}, {name});")
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C.replace("%FIELDS%", "\n  ".join(lines)))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True,
                               check=True).stdout.splitlines():
        T, f, v = line.split()
        got[(T, f)] = int(v)
    assert got[("ml_field_desc", "size")] == C.sizeof(ml.FieldDesc)
    assert got[("ml_field_params", "size")] == C.sizeof(ml.FieldParams)
    for T, S in (("ml_field_desc", ml.FieldDesc), ("ml_field_params", ml.FieldParams)):
        for name, _ in S._fields_:
            assert got[(T, name)] == getattr(S, name).offset, (T, name)


def test_smoke_field_meets_the_near_far_preconditions():
    """smoke() runs the mixed mode, which needs every ray inside the sheet's
    disc (the library refuses the field otherwise): the smoke field's ray
    rectangle, from the oracle's geometry, lies inside its disc."""
    import math
    import sys
    sys.path.insert(0, ROOT)
    import __graft_entry__ as entry
    import oracle
    w = entry.smoke_workload()
    g = oracle.geometry_of(w)
    cx, cy, r = w.sheet[:3]
    far = max(math.hypot(x - cx, y - cy) for x in (g.rx0, g.rx1) for y in (g.ry0, g.ry1))
    assert far < r
    assert 0.01 < g.kappa_star < 0.1 and g.n_rays > 100_000


def test_bench_traffic_check_ignores_comments():
    """bench.py keeps its measured DRAM traffic only for the kernel sources it
    was taken on, compared by a hash of their code: comment and spacing edits
    keep the hash, a changed operation does not; the committed sources match."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_for_test", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    a = "int f(int x)\n{\n    return x + 1;  // one\n}\n"
    b = "/* doc */\nint f(int x)\n{\n\n    return   x + 1;  // another comment\n}\n"
    c = "int f(int x)\n{\n    return x + 2;\n}\n"
    assert bench.code_hash(a) == bench.code_hash(b) != bench.code_hash(c)
    assert bench.traffic_per_launch(1e9) is not None
    # one measured figure per workload of the certified walk; none for the
    # per-ray walk or a workload that was not captured
    assert bench.traffic_per_launch(2e10) == pytest.approx(216.402944e6 + 269.967104e6)
    assert bench.traffic_per_launch(2e9, "fold") == pytest.approx(23.782144e6 + 512.0)
    assert bench.traffic_per_launch(1e9, "paper", "per_ray") is None
    assert bench.traffic_per_launch(1e9, "batched") is None


def test_bench_grid_flag_takes_an_optional_span_distance():
    """--grid fixes the level-1 size and level-2 subdivisions, and optionally
    the certified walk's lens distance ('inf': lens columns walked per ray)."""
    import sys
    import types
    bench = _bench_module()
    for grid, far in (("7.5,1.25,20,10", None), ("28.5,28,20,10,100", 100.0),
                      ("7.5,1.25,20,10,inf", 3.0e38)):
        argv = sys.argv
        try:
            sys.argv = ["bench.py", "--grid", grid]
            args = bench.parse()
        finally:
            sys.argv = argv
        w = types.SimpleNamespace()
        kw = bench.grid_kwargs(args, w)
        vals = [float(v) for v in grid.split(",")[:4]]
        assert w.l1 == (vals[0], vals[1]) and kw["l2_sub"] == (int(vals[2]), int(vals[3]))
        assert kw["tune"] is False and kw.get("span_far") == far


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_for_test", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench


def test_bench_peak_summary_and_baseline_records():
    """The fold step's peak summary divides as documented (crossings per
    theta_E of curve, mean mu at the peaks; empty bins report 0), and the CPU
    baseline taken from the parity stripe reports that run's rate."""
    import numpy as np
    bench = _bench_module()
    nb = len(bench.FOLD_DISTANCE_EDGES) - 1
    n = np.zeros(nb, np.uint64)
    s = np.zeros(nb, np.uint64)
    p = np.zeros(nb, np.uint64)
    n[2], s[2], p[2] = 4, 4000, 200
    p[3] = 50
    out = bench.fold_peak_summary((n, s, p), {"dpx": 0.02, "mu_per_count": 0.01})
    assert out["n_peaks"][2] == 4 and out["crossings_per_theta_e"][2] == 1.0
    assert out["mean_mu_peak"][2] == 10.0
    assert out["crossings_per_theta_e"][3] == 0.0 and out["mean_mu_peak"][3] == 0.0
    assert out["crossings_per_theta_e"][0] == 0.0
    assert len(out["edges_theta_e"]) == nb + 1

    class W:
        class lenses:
            n = 13000
    rec = bench.cpu_baseline_of((10_000_000, 12.5, 16, 1.0e11), W)
    assert rec["value"] == 800000.0 and rec["cores"] == 16 and rec["kind"] == "oracle"
    assert "10000000 consecutive rays" in rec["sample"]


def test_no_cpu_fallback_without_a_gpu_or_library(libpath, monkeypatch):
    """The product path fails loudly: without the built library the binding
    raises, and a valid descriptor on a machine without a usable GPU gets
    ML_ERR_CUDA and no field, never a result computed elsewhere."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes as C
    from paper_2308_14278_gb300 import inputs
    monkeypatch.setattr(ml, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        ml.load(os.path.join(ROOT, "no_such_dir", "libml.so"))
    lib = ml.load(libpath)
    d = ml.make_desc(inputs.small_map(0), precision=ml.PREC_MIXED)
    h = C.c_void_p()
    assert lib.ml_field_create(C.byref(d), None, C.byref(h)) == 3      # ML_ERR_CUDA
    assert h.value is None and lib.ml_last_error()


_CALLER_C = r"""
#include <stdio.h>
#include <string.h>
#include "ml.h"
int main(void)
{
    ml_field *f = (ml_field *)0;
    ml_field_desc d;
    memset(&d, 0, sizeof d);
    if (ml_abi_version() != ML_ABI_VERSION) return 1;
    if (ml_field_create((const ml_field_desc *)0, (void *)0, &f) != ML_ERR_INVALID_ARG) return 2;
    if (f != (ml_field *)0 || strlen(ml_last_error()) == 0) return 3;
    d.abi_version = ML_ABI_VERSION + 1;
    if (ml_field_create(&d, (void *)0, &f) != ML_ERR_INVALID_ARG) return 4;
    if (ml_field_destroy((ml_field *)0) != ML_OK) return 5;
    printf("%s\n", ml_last_error());
    return 0;
}
"""


def test_plain_c_program_links_and_calls_the_library(libpath, tmp_path):
    """The ABI is usable from C: a C11 program includes ml.h, links the
    shared library and gets the documented statuses (calls that need no GPU)."""
    src = tmp_path / "caller.c"
    src.write_text(_CALLER_C)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(libpath)
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(libpath),
                    "-Wl,-rpath," + libdir], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "abi_version" in r.stdout


@pytest.mark.parametrize("entry", ["ml_light_curves", "ml_light_curves_noalloc", "ml_map_light_curves"])
def test_light_curve_outputs_are_checked_before_any_call(libpath, entry):
    """A device output of the wrong dtype or too few values is refused in the
    binding, before the library would write n_tracks x n_samples float32s."""
    import torch
    tracks = np.array([[1.0, 1.0, 5.0, 5.0], [2.0, 2.0, 6.0, 3.0]])
    for out in (torch.empty((2, 16), dtype=torch.float64), torch.empty((2, 15), dtype=torch.float32)):
        with pytest.raises(ValueError):
            if entry == "ml_map_light_curves":
                ml.ml_map_light_curves(torch.zeros((8, 8)), tracks, 16, 0.5, out)
            else:
                getattr(ml, entry)(None, tracks, 16, 0.5, out)
    with pytest.raises(ValueError):
        ml.ml_light_curves(None, tracks, 16, 0.5, np.zeros((2, 15), np.float32))


def test_bench_clock_summary_keeps_the_timed_region(tmp_path):
    """The clock summary keeps the nvidia-smi samples stamped between the
    sampler's entry and exit (reporting their median SM clock and every
    throttle reason seen), and falls back to all samples when none is inside."""
    import datetime
    import time
    bench = _bench_module()
    c = bench.ClockSampler(0, str(tmp_path))
    c.proc = object()
    now = time.time()

    def st(t):
        return datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    rows = [(now - 1.0, 1500, "Not Active", "Not Active"), (now + 0.1, 2070, "Not Active", "Active"),
            (now + 0.2, 2070, "Not Active", "Not Active"), (now + 3.0, 1000, "Active", "Not Active")]
    with open(c.path, "w") as fh:
        for t, sm, hw, cap in rows:
            fh.write(f"{st(t)}, 0, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {cap}\n")
    c.t_in, c.t_out = now, now + 0.3
    s = c.summary()
    assert s["samples"] == 2 and s["in_timed_region"] and s["sm_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    c.t_in, c.t_out = now + 10.0, now + 11.0
    s = c.summary()
    assert s["samples"] == 4 and not s["in_timed_region"] and "hw_slowdown" in s["reasons"]
