"""CPU-only checks of the C ABI: the library loads, exports every declared symbol, and the
host-side argument checks behave (no compute call needs a GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "donof.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2004_06142_gb300 import build as b
    b.build()
    from paper_2004_06142_gb300 import binding
    return binding.lib()


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"\b(donof_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "donof_energy_lagrangian" in names and "donof_energy_backward" in names
    for n in names:
        assert hasattr(lib, n), n


def test_enums_match_binding():
    from paper_2004_06142_gb300 import binding
    src = open(HEADER).read()
    def val(name):
        return int(re.search(rf"\b{name}\s*=\s*(-?\d+)", src).group(1))
    assert val("DONOF_PNOF5") == binding.PNOF5
    assert val("DONOF_PNOF7") == binding.PNOF7
    assert val("DONOF_PNOF7S") == binding.PNOF7S
    assert val("DONOF_B_PACKED") == binding.B_PACKED
    assert val("DONOF_MIXED") == binding.MIXED
    for code, text in binding.STATUS.items():
        assert binding.donof_status_string(code) == text


def test_struct_layout_matches_header(lib):
    from paper_2004_06142_gb300 import binding
    assert ctypes.sizeof(binding.donof_problem) == 8 * 4 + 8


def test_workspace_size_and_argument_checks(lib):
    from paper_2004_06142_gb300 import binding as b
    small = b.donof_workspace_size(b.make_problem(24, 96, 5, 1))
    assert small > 0
    mixed = b.donof_workspace_size(b.make_problem(24, 96, 5, 1, precision=b.MIXED))
    assert mixed > small
    budget = b.donof_workspace_size(b.make_problem(500, 2000, 20, 3, x_budget_bytes=1 << 26))
    full = b.donof_workspace_size(b.make_problem(500, 2000, 20, 3))
    assert budget < full
    bad = [
        b.make_problem(0, 96, 5, 1),
        b.make_problem(24, 96, 5, 1, functional=6),
        b.make_problem(24, 96, 13, 1),           # nact > nbf
        b.make_problem(24, 96, 5, 1, b_layout=3),
        b.make_problem(24, 96, 5, 1, precision=2),
    ]
    for p in bad:
        with pytest.raises(b.DonofError) as e:
            b.donof_workspace_size(p)
        assert e.value.code == -1
    with pytest.raises(b.DonofError) as e:       # nact 300 > 256 on the tensor-core path
        b.donof_workspace_size(b.make_problem(400, 100, 100, 2, precision=b.MIXED))
    assert e.value.code == -7


def test_entry_points_reject_null_workspace(lib):
    from paper_2004_06142_gb300 import binding as b
    p = b.make_problem(24, 96, 5, 1)
    rc = lib.donof_prepare_B(ctypes.byref(p), ctypes.c_void_p(256), None, 0, None)
    assert rc == -4
    E = ctypes.c_void_p(256)
    rc = lib.donof_energy_lagrangian(ctypes.byref(p), E, E, E, E, E, None, 0, E, None, None, None)
    assert rc == -4
    rc = lib.donof_energy_lagrangian(ctypes.byref(p), None, E, E, E, E, E, 0, E, None, None, None)
    assert rc == -1


def test_eigensolver_and_host_entry_argument_checks(lib):
    """Host-side argument checks of the eigensolver and of the host-buffer build: refused
    before any device work (the pointers here are never dereferenced)."""
    from paper_2004_06142_gb300 import binding as b
    nb = ctypes.c_size_t(0)
    assert lib.donof_eigh_workspace_size(0, ctypes.byref(nb)) == -1
    assert lib.donof_eigh_workspace_size(4097, ctypes.byref(nb)) == -1
    assert lib.donof_eigh_workspace_size(10, ctypes.byref(nb)) == 0
    assert nb.value >= 3 * 10 * 10 * 8
    assert lib.donof_orbital_update_workspace_size(4097, ctypes.byref(nb)) == -1
    X = ctypes.c_void_p(256)
    assert lib.donof_eigh(0, X, X, X, X, 1 << 20, None) == -1
    assert lib.donof_eigh(10, None, X, X, X, 1 << 20, None) == -1
    assert lib.donof_eigh(10, X, X, X, None, 0, None) == -4
    assert lib.donof_eigh(10, X, X, X, X, 16, None) == -4
    p = b.make_problem(24, 96, 5, 1)
    assert lib.donof_host_staging_size(ctypes.byref(p), ctypes.byref(nb)) == 0
    assert nb.value >= 3 * 24 * 24 * 8
    bad = b.make_problem(0, 96, 5, 1)
    assert lib.donof_host_staging_size(ctypes.byref(bad), ctypes.byref(nb)) == -1
    args = [X, X, X, X, X, X, 1 << 20, X, 1 << 20, X, None, None, None, None]
    # NULL host orbitals; a staging buffer smaller than donof_host_staging_size
    a1 = list(args)
    a1[2] = None
    assert lib.donof_energy_lagrangian_host(ctypes.byref(p), *a1) == -1
    a2 = list(args)
    a2[8] = 64
    assert lib.donof_energy_lagrangian_host(ctypes.byref(p), *a2) == -4


def test_injected_workspace_allocation_failure(lib, monkeypatch):
    """Host-side fault injection: with DONOF_INJECT_ALLOC_FAILURE=1 every workspace the
    binding would allocate fails as an allocation failure does, before any device is
    touched, and surfaces as DonofError with the workspace status."""
    from paper_2004_06142_gb300 import binding as b
    monkeypatch.setenv("DONOF_INJECT_ALLOC_FAILURE", "1")
    with pytest.raises(b.DonofError) as e:
        b.Builder(24, 96, 5, 1)
    assert e.value.code == b.ERR_WORKSPACE
    assert "injected" in str(e.value)
    with pytest.raises(b.DonofError) as e:
        b.alloc_workspace(1 << 20, "cpu")
    assert e.value.code == b.ERR_WORKSPACE
    monkeypatch.delenv("DONOF_INJECT_ALLOC_FAILURE")
    assert b.alloc_workspace(1 << 10, "cpu").numel() == 1 << 10
