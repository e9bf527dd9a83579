"""Host-side parts of the measurement driver: kernel-name shortening of the launch list, and the
in-process CUPTI activity collector (csrc/launch_trace.cpp) building, loading and reporting no
records before it is started (no GPU needed)."""
import shutil

import pytest

from paper_2508_19138_gb300.kernel_driver import _load_tracer, _short_name


@pytest.mark.parametrize("raw,short", [
    ("void bt::(anonymous namespace)::split_mma_kernel<112, 0, false>(CUtensorMap, CUtensorMap, "
     "CUtensorMap, bt::(anonymous namespace)::MmaParams)", "split_mma_kernel<112, 0, false>"),
    ("void bt::<unnamed>::gj_panel_cluster_kernel<8>(int, int, int, double2*, long long, int*, int*, const int*)",
     "gj_panel_cluster_kernel<8>"),
    ("void (anonymous namespace)::zgemm_kernel<0, 0, 1, 32>(int, int, int)", "zgemm_kernel<0, 0, 1, 32>"),
    ("memcpy", "memcpy"),
    ("Memcpy DtoH (Device -> Pinned)", "Memcpy DtoH"),
])
def test_short_names(raw, short):
    assert _short_name(raw) == short


def test_tracer_builds_and_loads_without_records():
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    try:
        lib = _load_tracer()
    except Exception as exc:  # the toolkit's libcupti or its headers are not installed here
        pytest.skip(f"CUPTI collector unavailable: {exc}")
    assert lib.bt_trace_count() == 0
    import ctypes as C
    name = C.create_string_buffer(64)
    t0, t1 = C.c_ulonglong(0), C.c_ulonglong(0)
    assert lib.bt_trace_get(0, name, 64, C.byref(t0), C.byref(t1)) == -1
