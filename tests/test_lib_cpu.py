"""Host-side checks of the CUDA library that need no GPU: it builds, loads, and exports every
entry point that include/lat.h declares (no compute calls are made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            src = open(os.path.join(ROOT, "include", hdr)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(lat_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1508_02899_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("lat_init", "lat_set_flow", "lat_step", "lat_moments", "lat_free"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.lat_strerror.restype = ctypes.c_char_p
    assert lib.lat_strerror(0) == b"ok"
    assert b"stability" in lib.lat_strerror(2)


def test_binding_marshals_structs_like_the_header():
    from paper_1508_02899_gb300 import lat
    # lat_grid: 5 ints then 4 doubles (8-byte aligned); lat_flow: pointers at 8-byte offsets
    assert ctypes.sizeof(lat.LatGrid) == 56
    assert lat.LatGrid.L.offset == 24
    assert ctypes.sizeof(lat.LatInstance) == 40
    assert lat.LatFlow.field.offset == 8 and lat.LatFlow.k.offset == 24
    assert ctypes.sizeof(lat.LatFlow) == 64


def test_committed_profiles_carry_their_roofline_inputs():
    """Every ncu summary that states a traffic figure also states the units it covers and the
    source hash it was taken on, in the form bench.py reads."""
    import bench
    prof = os.path.join(bench.ROOT, "profiles")
    found = 0
    for name in sorted(os.listdir(prof)):
        vals = bench.parse_profile(open(os.path.join(prof, name)).read())
        if "traffic_bytes_per_launch" in vals:
            found += 1
            assert float(vals["traffic_bytes_per_launch"]) > 0
            assert float(vals["units_per_launch"]) > 0
            assert re.fullmatch(r"[0-9a-f]{16}", vals["source_sha256"])
    assert found >= 3


def test_timed_workloads_have_current_traffic_figures():
    """The ncu summary of the dominant kernel of every timed workload was taken on the current
    sources, so that bench.py reports its DRAM
    traffic (a summary left behind by a kernel change reads as a null traffic figure)."""
    import bench
    for workload in ("ensemble", "ensemble_koren", "2d", "2d_f16", "2d_bf16", "2d_learned"):
        prof, src = bench.KERNEL_PROFILES[workload]
        assert bench.profile_traffic(prof, src) is not None, (workload, bench.source_hash(src))


def test_library_leaves_no_internal_symbol_undefined(libpath):
    """Every function of the library's own namespace that one translation unit calls is defined
    in another (a shared library links with undefined symbols and would fail only when loaded
    on the GPU machine)."""
    import subprocess
    out = subprocess.run(["nm", "-D", "--undefined-only", "-C", libpath], capture_output=True,
                         text=True, check=True).stdout
    bad = [l for l in out.splitlines() if "lat::" in l or " lat_" in l]
    assert not bad, bad
