"""The C-ABI library loads without a GPU and exports what include/lbc.h
declares; host-only entry points behave as documented.  No compute calls."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1406_2211_gb300 import builder, lbc
    builder.build()
    return lbc.library(build_if_missing=False)


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbc_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = _declared_functions()
    assert "lbc_box_step" in names and "lbc_box_create" in names
    assert len(names) >= 20


def test_every_declared_symbol_is_exported(lib):
    raw = C.CDLL(lib._name)
    missing = [n for n in _declared_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_constants_match_header():
    from paper_1406_2211_gb300 import lbc
    text = open(HEADER).read()
    defs = dict(re.findall(r"#define\s+(LBC_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text))
    assert defs, "no constants parsed"
    for name, val in defs.items():
        assert hasattr(lbc, name), name
        assert getattr(lbc, name) == int(val), name


def test_descriptor_sizes_match(lib):
    from paper_1406_2211_gb300 import lbc
    sizes = (C.c_size_t * 3)()
    lib.lbc_desc_sizes(sizes)
    assert tuple(sizes) == (C.sizeof(lbc.lbc_lattice_desc), C.sizeof(lbc.lbc_coupling_desc),
                            C.sizeof(lbc.lbc_particles_desc))


def test_abi_version_and_status_strings(lib):
    assert lib.lbc_abi_version() == 2
    assert lib.lbc_status_string(0) == b"ok"
    assert lib.lbc_status_string(-2) == b"caller memory too small"
    assert lib.lbc_status_string(99) == b"unknown status"


def test_bytes_required_host_only(lib):
    from paper_1406_2211_gb300 import lbc
    n = C.c_size_t()
    lat = lbc.lattice_desc(32, 24, 16, collision="mrt", tau=1.0, storage="f32")
    cpl = lbc.coupling_desc("fc", 2, "trilinear", gamma=1.0)
    assert lib.lbc_box_bytes_required(C.byref(lat), C.byref(cpl), 100, 99, C.byref(n)) == 0
    pops = 2 * 19 * 32 * 24 * 16 * 4
    assert n.value >= pops
    # FP64 storage doubles the population bytes
    lat64 = lbc.lattice_desc(32, 24, 16, storage="f64")
    n64 = C.c_size_t()
    none = lbc.coupling_desc()
    assert lib.lbc_box_bytes_required(C.byref(lat64), C.byref(none), 0, 0, C.byref(n64)) == 0
    assert n64.value >= 2 * pops
    # ragged rows are padded to 32-byte multiples
    lat_r = lbc.lattice_desc(13, 7, 5, storage="f32")
    nr = C.c_size_t()
    assert lib.lbc_box_bytes_required(C.byref(lat_r), C.byref(none), 0, 0, C.byref(nr)) == 0
    assert nr.value >= 2 * 19 * 16 * 7 * 5 * 4


@pytest.mark.parametrize("field,value", [("nx", 0), ("tau", 0.5), ("storage", 9),
                                         ("collision", 3), ("rho0", 0.0)])
def test_invalid_lattice_rejected(lib, field, value):
    from paper_1406_2211_gb300 import lbc
    lat = lbc.lattice_desc(8, 8, 8)
    setattr(lat, field, value)
    n = C.c_size_t()
    assert lib.lbc_box_bytes_required(C.byref(lat), None, 0, 0, C.byref(n)) == lbc.LBC_ERR_ARG


def test_invalid_coupling_rejected(lib):
    from paper_1406_2211_gb300 import lbc
    lat = lbc.lattice_desc(8, 8, 8)
    n = C.c_size_t()
    bad = [lbc.coupling_desc("fc", 3), lbc.coupling_desc("fc", 2, gamma=0.0),
           lbc.coupling_desc("ibm", 2, split="outside", substeps=2),
           lbc.coupling_desc("fc", 1, split="inside", substeps=2)]
    for cpl in bad:
        assert lib.lbc_box_bytes_required(C.byref(lat), C.byref(cpl), 4, 0,
                                          C.byref(n)) == lbc.LBC_ERR_ARG


def test_create_rejects_small_or_misaligned_arena(lib):
    """Argument checks happen before any device work."""
    from paper_1406_2211_gb300 import lbc
    lat = lbc.lattice_desc(8, 8, 8)
    h = C.c_void_p()
    assert lib.lbc_box_create(C.byref(lat), None, 0, 0, C.c_void_p(256), 16, None,
                              C.byref(h)) == lbc.LBC_ERR_OOM
    assert lib.lbc_box_create(C.byref(lat), None, 0, 0, C.c_void_p(8), 1 << 30, None,
                              C.byref(h)) == lbc.LBC_ERR_ARG


def test_product_package_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_1406_2211_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\b(import|from)\s+oracle\b", text), f
                assert "oracle/" not in text, f


def test_batch_bytes_required_host_only(lib):
    n1 = lib.lbc_batch_bytes_required(1)
    n8 = lib.lbc_batch_bytes_required(8)
    # tables scale with the slots (regions are padded to 256 bytes)
    assert n1 > 0 and 7 * n1 < n8 <= 8 * n1
    assert lib.lbc_batch_bytes_required(0) == 0
    assert lib.lbc_batch_bytes_required(2000) == 0  # above the 1024-slot limit


def test_null_handles_are_rejected(lib):
    from paper_1406_2211_gb300 import lbc
    out = C.c_void_p()
    fin = (C.c_void_p * 1)()
    nfin, done, n = C.c_int32(), C.c_int64(), C.c_int64()
    assert lib.lbc_batch_create(0, None, 0, C.byref(out)) == lbc.LBC_ERR_ARG
    assert lib.lbc_batch_add(None, None, 1) == lbc.LBC_ERR_ARG
    assert lib.lbc_batch_remove(None, None) == lbc.LBC_ERR_ARG
    assert lib.lbc_batch_remaining(None, None, C.byref(n)) == lbc.LBC_ERR_ARG
    assert lib.lbc_batch_advance(None, 1, None, fin, C.byref(nfin), C.byref(done)) == lbc.LBC_ERR_ARG
    assert lib.lbc_batch_size(None) == -1
    assert lib.lbc_batch_destroy(None) == lbc.LBC_ERR_ARG
    assert lib.lbc_box_get_stress(None, None, None) == lbc.LBC_ERR_ARG
    assert lib.lbc_box_autotune(None, None, None, None) == lbc.LBC_ERR_ARG
    assert lib.lbc_box_set_option(None, lbc.LBC_OPT_NODE_MOMENTS, 1) == lbc.LBC_ERR_ARG
    assert lib.lbc_box_get_option(None, lbc.LBC_OPT_NODE_MOMENTS, C.byref(n)) == lbc.LBC_ERR_ARG
    assert lib.lbc_box_set_thermal(None, 1e-4, 1) == lbc.LBC_ERR_ARG
