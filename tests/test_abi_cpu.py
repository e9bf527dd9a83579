"""CPU-side checks of the C ABI: the library builds, loads and exports every entry point that
include/bt_selinv.h declares; host-only argument validation (no GPU work is issued)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"BT_API\s+[\w\s\*]+?\b(bt_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2508_19138_gb300 import _native
    from paper_2508_19138_gb300 import build
    build.build()
    return _native.load()


def test_header_declares_entry_points():
    names = declared_entry_points()
    assert "bt_selinv_create" in names and "bt_selinv_solve" in names and "bt_selinv_destroy" in names
    assert len(names) >= 14


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_covers_every_entry_point():
    import paper_2508_19138_gb300 as pkg
    from paper_2508_19138_gb300 import _native
    for name in declared_entry_points():
        assert name in _native.SIGNATURES, name
        assert hasattr(pkg, name), f"binding lacks {name}"


def test_workspace_sizes_host_logic(lib):
    import paper_2508_19138_gb300 as pkg
    d = pkg.make_desc(8, 32, 64)
    n1 = pkg.bt_selinv_workspace_bytes(d)
    d2 = pkg.make_desc(8, 32, 128)
    assert pkg.bt_selinv_workspace_bytes(d2) > n1 > 0
    # blocked inverse needs pivots + panel copy, small inverse none
    assert pkg.bt_zinv_workspace_bytes(32, 10) == 0
    assert pkg.bt_zinv_workspace_bytes(416, 10) >= 10 * 416 * 4 + 10 * 16 * 416 * 16
    assert pkg.bt_decimate_workspace_bytes(32, 4) >= 10 * 4 * 32 * 32 * 16


@pytest.mark.parametrize("kw,needle", [
    (dict(nb=0), "nb"), (dict(bs=0), "bs"), (dict(max_energies=0), "max_energies"),
    (dict(nb=1, obc=True), "nb >= 2"), (dict(system=1, obc=True, obc_memo=True), "G system"),
    (dict(precision=1, split_slices=12), "split_slices"), (dict(kT=0.0), "kT"),
])
def test_create_rejects_bad_descriptors_on_host(lib, kw, needle):
    import paper_2508_19138_gb300 as pkg
    base = dict(nb=4, bs=8, max_energies=4, system=0, precision=0, split_slices=0, obc=True, kT=0.025)
    base.update(kw)
    d = pkg.make_desc(base["nb"], base["bs"], base["max_energies"], base["system"], base["precision"],
                      base["split_slices"], True, base["obc"], 1e-6, base["kT"], obc_memo=base.get("obc_memo", False))
    with pytest.raises(pkg.BTError) as ei:
        pkg.bt_selinv_create(d, stream=0)
    assert ei.value.status == pkg.BT_ERR_INVALID_ARG
    assert needle in str(ei.value)


def test_graph_mode_validation_on_host(lib):
    import paper_2508_19138_gb300 as pkg
    d = pkg.make_desc(4, 8, 4, obc=True, obc_memo=True, graph=True)
    with pytest.raises(pkg.BTError) as ei:
        pkg.bt_selinv_create(d, stream=0)
    assert ei.value.status == pkg.BT_ERR_INVALID_ARG and "exclusive" in str(ei.value)
    d = pkg.make_desc(4, 8, 4)
    d.graph = 2
    with pytest.raises(pkg.BTError) as ei:
        pkg.bt_selinv_create(d, stream=0)
    assert "graph" in str(ei.value)


def test_budget_rejection_on_host(lib):
    import paper_2508_19138_gb300 as pkg
    d = pkg.make_desc(40, 416, 64, hbm_budget_bytes=1 << 20)
    with pytest.raises(pkg.BTError) as ei:
        pkg.bt_selinv_create(d, stream=0)
    assert ei.value.status == pkg.BT_ERR_BUDGET


def test_primitive_argument_checks_on_host(lib):
    # invalid ops / leading dimensions are rejected before any launch
    assert lib.bt_zgemm_batched(4, 4, 4, 1.0, 0.0, None, 4, 0, 7, None, 4, 0, 0, 0.0, 0.0, None, 4, 0, 1, None) == 1
    assert lib.bt_zgemm_batched(4, 4, 4, 1.0, 0.0, C.c_void_p(16), 2, 0, 0, C.c_void_p(16), 4, 0, 0, 0.0, 0.0,
                                C.c_void_p(16), 4, 0, 1, None) == 1
    assert lib.bt_zinv_batched(-1, None, 0, 1, None, None, 0, None) == 1


def test_packed_upper_layout_formula():
    """BT_LAYOUT_PACKED_UPPER as the header states it: entry (r, c >= r) at r bs - r (r - 1) / 2 + (c - r);
    unpack_upper rebuilds the anti-Hermitian block from it."""
    import numpy as np
    from gpu_util import unpack_upper
    bs = 7
    rng = np.random.default_rng(3)
    X = rng.standard_normal((bs, bs)) + 1j * rng.standard_normal((bs, bs))
    A = 0.5 * (X - X.conj().T)
    packed = np.zeros(bs * (bs + 1) // 2, dtype=np.complex128)
    for r in range(bs):
        for c in range(r, bs):
            packed[r * bs - r * (r - 1) // 2 + (c - r)] = A[r, c]
    assert np.array_equal(unpack_upper(packed, bs), A)
