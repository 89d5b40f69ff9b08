"""The C ABI library loads, exports every function include/chemora.h
declares, and validates arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1410_1764_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "chemora.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chemora_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(N.LIB_PATH):
        import importlib.util
        spec = importlib.util.spec_from_file_location("b", os.path.join(ROOT, "paper_1410_1764_gb300", "build.py"))
        m = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(m)
        m.build()
    return N.lib()


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(N.SIGNATURES), set(names) ^ set(N.SIGNATURES)


def test_grid_validation(L):
    h = ctypes.c_void_p()
    assert L.chemora_grid_create(0, 4, 4, 2, 2, 0.1, ctypes.byref(h)) == N.EINVAL
    assert b"sizes" in L.chemora_last_error()
    assert L.chemora_grid_create(4, 4, 4, 2, 2, -1.0, ctypes.byref(h)) == N.EINVAL
    assert L.chemora_grid_create(4, 4, 4, 2, 2, float("nan"), ctypes.byref(h)) == N.EINVAL
    assert L.chemora_grid_create(4, 4, 4, 2, 2, 0.1, None) == N.EINVAL
    assert L.chemora_grid_create(4, 5, 6, 2, 2, 0.1, ctypes.byref(h)) == N.OK
    sy, sz, sv = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    assert L.chemora_grid_layout(h, ctypes.byref(sy), ctypes.byref(sz), ctypes.byref(sv)) == N.OK
    assert (sy.value, sz.value, sv.value) == (8, 8 * 9, 8 * 9 * 10)
    L.chemora_destroy(h)


def test_system_validation(L):
    g = ctypes.c_void_p()
    assert L.chemora_grid_create(8, 8, 8, 2, 2, 0.1, ctypes.byref(g)) == N.OK
    s = ctypes.c_void_p()
    assert L.chemora_system_create(g, N.BSSN, None, ctypes.byref(s)) == N.EINVAL  # nvars 2
    assert L.chemora_system_create(g, 99, None, ctypes.byref(s)) == N.EINVAL
    bad = N.Params(0.1, 2.0, 7, 0)
    assert L.chemora_system_create(g, N.WAVE, ctypes.byref(bad), ctypes.byref(s)) == N.EINVAL
    assert L.chemora_system_create(g, N.WAVE, None, ctypes.byref(s)) == N.OK
    # host-side checks before any device work
    assert L.chemora_rk4_step(s, None, 0.1, 1, None) == N.EINVAL
    assert L.chemora_rk4_step(s, ctypes.c_void_p(8), 0.1, -1, None) == N.EINVAL
    assert L.chemora_rk4_step(s, ctypes.c_void_p(8), float("inf"), 1, None) == N.EINVAL
    assert L.chemora_rhs(s, ctypes.c_void_p(8), ctypes.c_void_p(8), None) == N.EINVAL
    assert L.chemora_system_set_speed(s, ctypes.c_void_p(8), None) == N.EINVAL  # not var-c
    assert L.chemora_rhs(g, ctypes.c_void_p(8), ctypes.c_void_p(16), None) == N.EINVAL  # wrong handle
    L.chemora_destroy(s)
    g3 = ctypes.c_void_p()
    assert L.chemora_grid_create(8, 8, 8, 2, 2, 0.1, ctypes.byref(g3)) == N.OK
    sv = ctypes.c_void_p()
    assert L.chemora_system_create(g3, N.WAVE_VARC, None, ctypes.byref(sv)) == N.OK
    assert L.chemora_rk4_step(sv, ctypes.c_void_p(8), 0.1, 1, None) == N.EINVAL  # no speed yet
    L.chemora_destroy(sv)
    L.chemora_destroy(g3)
    L.chemora_destroy(g)
    L.chemora_destroy(None)


def test_opcounts_match_generator(L):
    import json
    counts = json.load(open(os.path.join(ROOT, "paper_1410_1764_gb300", "csrc", "generated",
                                         "opcounts.json")))
    for kind, key in ((N.WAVE, "wave"), (N.WAVE_VARC, "wave_varc"), (N.BSSN, "bssn")):
        i, f = ctypes.c_int64(), ctypes.c_int64()
        assert L.chemora_opcount(kind, ctypes.byref(i), ctypes.byref(f)) == N.OK
        assert (i.value, f.value) == (counts[key]["fp64_instructions"], counts[key]["flops"])


def test_generated_sources_up_to_date():
    from paper_1410_1764_gb300.gen import __main__ as G
    files = G.render()
    for name, text in files.items():
        path = os.path.join(G.OUT, name)
        assert open(path).read() == text, "regenerate: python -m paper_1410_1764_gb300.gen"


def test_variant_queries(L):
    for kind in (N.WAVE, N.WAVE_VARC, N.BSSN):
        assert L.chemora_variant_count(kind) >= 4
    assert L.chemora_variant_count(42) == 0
    g, s = ctypes.c_void_p(), ctypes.c_void_p()
    assert L.chemora_grid_create(8, 8, 8, 24, 3, 0.1, ctypes.byref(g)) == N.OK
    assert L.chemora_system_create(g, N.BSSN, None, ctypes.byref(s)) == N.OK
    v, tx, ty = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert L.chemora_system_variant(s, -1, ctypes.byref(v), ctypes.byref(tx), ctypes.byref(ty)) == N.OK
    assert (v.value, tx.value, ty.value) == (0, 32, 4)
    assert L.chemora_system_variant(s, 2, ctypes.byref(v), ctypes.byref(tx), ctypes.byref(ty)) == N.OK
    assert v.value == 2
    assert L.chemora_system_variant(s, 99, None, None, None) == N.EINVAL
    L.chemora_destroy(s)
    L.chemora_destroy(g)


def test_order_validation(L):
    g = ctypes.c_void_p()
    s = ctypes.c_void_p()
    assert L.chemora_grid_create(8, 8, 8, 2, 2, 0.1, ctypes.byref(g)) == N.OK
    p6 = N.Params(0.1, 2.0, 0, 0, 6)
    assert L.chemora_system_create(g, N.WAVE, ctypes.byref(p6), ctypes.byref(s)) == N.EINVAL  # ghosts
    p5 = N.Params(0.1, 2.0, 0, 0, 5)
    assert L.chemora_system_create(g, N.WAVE, ctypes.byref(p5), ctypes.byref(s)) == N.EINVAL  # odd
    p2 = N.Params(0.1, 2.0, 0, 0, 2)
    assert L.chemora_system_create(g, N.WAVE, ctypes.byref(p2), ctypes.byref(s)) == N.OK
    L.chemora_destroy(s)
    g3, g5 = ctypes.c_void_p(), ctypes.c_void_p()
    assert L.chemora_grid_create(8, 8, 8, 24, 3, 0.1, ctypes.byref(g3)) == N.OK
    assert L.chemora_system_create(g3, N.BSSN, ctypes.byref(p6), ctypes.byref(s)) == N.EINVAL
    assert L.chemora_grid_create(8, 8, 8, 5, 4, 0.1, ctypes.byref(g5)) == N.OK
    p8 = N.Params(0.1, 2.0, 0, 0, 8)
    assert L.chemora_system_create(g5, N.WAVE1, ctypes.byref(p8), ctypes.byref(s)) == N.OK
    L.chemora_destroy(s)
    for h in (g, g3, g5):
        L.chemora_destroy(h)


def test_specialize_host_checks(L):
    g, s = ctypes.c_void_p(), ctypes.c_void_p()
    assert L.chemora_grid_create(8, 8, 8, 2, 2, 0.1, ctypes.byref(g)) == N.OK
    assert L.chemora_system_create(g, N.WAVE, None, ctypes.byref(s)) == N.OK
    secs = ctypes.c_double(-1.0)
    assert L.chemora_system_specialize(s, 1, None, ctypes.byref(secs)) == N.EUNSUPPORTED
    assert b"BSSN" in L.chemora_last_error()
    assert secs.value == 0.0
    assert L.chemora_system_specialize(s, 0, None, None) == N.OK
    assert L.chemora_system_specialize(g, 1, None, None) == N.EINVAL   # a grid, not a system
    L.chemora_destroy(s)
    L.chemora_destroy(g)


def test_specialised_source_compiles_with_nvrtc(L, tmp_path):
    """The run-time specialised BSSN stage source (x/y-sharing body, one
    kernel per RK stage mode) compiles for sm_103a with NVRTC, which needs no
    GPU; on a host without a device the load then fails with ECUDA, after the
    cubins reached the cache."""
    g, s = ctypes.c_void_p(), ctypes.c_void_p()
    assert L.chemora_grid_create(64, 64, 16, 24, 3, 1.0 / 64, ctypes.byref(g)) == N.OK
    assert L.chemora_system_create(g, N.BSSN, None, ctypes.byref(s)) == N.OK
    v, tx, ty = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    xy8 = 15                                            # a 32 x 8 x/y-sharing shape
    assert L.chemora_system_variant(s, xy8, ctypes.byref(v), ctypes.byref(tx), ctypes.byref(ty)) == N.OK
    assert (tx.value, ty.value) == (32, 8)
    secs = ctypes.c_double()
    rc = L.chemora_system_specialize(s, 1, str(tmp_path).encode(), ctypes.byref(secs))
    try:
        if rc == N.EUNSUPPORTED:
            pytest.skip(L.chemora_last_error().decode())
        assert rc in (N.OK, N.ECUDA), L.chemora_last_error()
        if rc == N.ECUDA:
            assert b"cudaLibraryLoadData" in L.chemora_last_error()
        cubins = sorted(tmp_path.glob("*.cubin"))
        assert len(cubins) == 5
        for c in cubins:
            assert c.read_bytes()[:4] == b"\x7fELF"
    finally:
        L.chemora_destroy(s)
        L.chemora_destroy(g)


def test_variant_info(L):
    tx, ty, mb, sh = (ctypes.c_int() for _ in range(4))
    n = L.chemora_variant_count(N.BSSN)
    seen = set()
    for v in range(n):
        assert L.chemora_variant_info(N.BSSN, v, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(mb),
                                      ctypes.byref(sh)) == N.OK
        assert tx.value * ty.value <= 1024 and mb.value >= 1 and sh.value in (0, 1, 2)
        if sh.value == 2:
            assert tx.value == 32 and ty.value >= 5      # the prologue's halo rows need 5 warp rows
        seen.add(sh.value)
    assert seen == {0, 1, 2}
    assert L.chemora_variant_info(N.BSSN, 0, None, None, None, None) == N.OK
    assert L.chemora_variant_info(N.BSSN, n, None, None, None, None) == N.EINVAL
    assert L.chemora_variant_info(77, 0, None, None, None, None) == N.EINVAL


def test_specialise_recovers_from_a_damaged_cache(L, tmp_path):
    """Cubins in the cache that are damaged (an ELF header and nothing else)
    are compiled again; on a host without a device the load still fails with
    ECUDA, with fresh cubins in the cache."""
    def spec():
        g, s = ctypes.c_void_p(), ctypes.c_void_p()
        assert L.chemora_grid_create(32, 32, 8, 24, 3, 1.0 / 32, ctypes.byref(g)) == N.OK
        assert L.chemora_system_create(g, N.BSSN, None, ctypes.byref(s)) == N.OK
        rc = L.chemora_system_specialize(s, 1, str(tmp_path).encode(), None)
        L.chemora_destroy(s)
        L.chemora_destroy(g)
        return rc
    rc = spec()
    if rc == N.EUNSUPPORTED:
        pytest.skip("NVRTC not available")
    cubins = sorted(tmp_path.glob("*.cubin"))
    assert len(cubins) == 5
    for c in cubins:
        c.write_bytes(b"\x7fELF" + b"\0" * 12)
    rc2 = spec()
    assert rc2 == rc
    for c in cubins:
        assert c.stat().st_size > 1000


def test_edge_sizes_rejected_on_the_host(L):
    """Empty, oversized and out-of-range inputs are refused before any device
    work: grid extents beyond the launch limits or the 2^40-double state
    cap, empty or oversized patch lists, AMR boxes outside the coarse grid."""
    h = ctypes.c_void_p()
    assert L.chemora_grid_create(65535 * 32 + 1, 4, 4, 2, 2, 0.1, ctypes.byref(h)) == N.EINVAL
    assert L.chemora_grid_create(4, 65535 * 4 + 1, 4, 2, 2, 0.1, ctypes.byref(h)) == N.EINVAL
    assert L.chemora_grid_create(4, 4, 65536, 2, 2, 0.1, ctypes.byref(h)) == N.EINVAL
    assert L.chemora_grid_create(16384, 16384, 16384, 24, 3, 0.1, ctypes.byref(h)) == N.EINVAL
    assert b"large" in L.chemora_last_error() or b"limit" in L.chemora_last_error()
    assert L.chemora_grid_create(1, 1, 1, 2, 2, 0.1, ctypes.byref(h)) == N.OK   # one point is a grid
    L.chemora_destroy(h)
    b = ctypes.c_void_p()
    dims = (ctypes.c_int * 3)(16, 16, 16)
    assert L.chemora_patches_create(0, dims, 3, 0.1, N.BSSN, None, ctypes.byref(b)) == N.EINVAL
    assert L.chemora_patches_create(1, None, 3, 0.1, N.BSSN, None, ctypes.byref(b)) == N.EINVAL
    for bad in ((0, 16, 16), (16, 5000, 16)):
        d = (ctypes.c_int * 3)(*bad)
        assert L.chemora_patches_create(1, d, 3, 0.1, N.BSSN, None, ctypes.byref(b)) == N.EINVAL
    assert L.chemora_patches_create(1, dims, 3, 0.0, N.BSSN, None, ctypes.byref(b)) == N.EINVAL
    assert L.chemora_patches_create(1, dims, 3, 0.1, N.WAVE_VARC, None, ctypes.byref(b)) == N.EINVAL
    assert L.chemora_patches_set_time_limit(None, 1.0) == N.EINVAL
    a = ctypes.c_void_p()
    lo, hi = (ctypes.c_int * 3)(8, 8, 8), (ctypes.c_int * 3)(24, 24, 24)
    assert L.chemora_amr_create(0, lo, hi, 0.1, ctypes.byref(a)) == N.EINVAL
    assert L.chemora_amr_create(32, None, hi, 0.1, ctypes.byref(a)) == N.EINVAL
    out_box = (ctypes.c_int * 3)(8, 8, 40)
    assert L.chemora_amr_create(32, lo, out_box, 0.1, ctypes.byref(a)) == N.EINVAL
    empty_box = (ctypes.c_int * 3)(8, 8, 8)
    assert L.chemora_amr_create(32, lo, empty_box, 0.1, ctypes.byref(a)) == N.EINVAL
    # several boxes: BSSN margins (5 <= lo, hi <= nc - 6), overlap, kind, count
    nc3 = (ctypes.c_int * 3)(32, 30, 28)
    two_lo = (ctypes.c_int * 6)(5, 5, 5, 12, 5, 5)
    two_hi = (ctypes.c_int * 6)(10, 10, 10, 20, 10, 10)
    bad_lo = (ctypes.c_int * 6)(4, 5, 5, 12, 5, 5)  # 4 < 5
    assert L.chemora_amr_create_boxes(N.BSSN, nc3, 2, bad_lo, two_hi, 0.1, None, ctypes.byref(a)) == N.EINVAL
    bad_hi = (ctypes.c_int * 6)(5, 5, 5, 12, 5, 5)
    bad_hi_v = (ctypes.c_int * 6)(10, 10, 10, 20, 10, 23)  # 23 > 28 - 6
    assert L.chemora_amr_create_boxes(N.BSSN, nc3, 2, bad_hi, bad_hi_v, 0.1, None, ctypes.byref(a)) == N.EINVAL
    ov_lo = (ctypes.c_int * 6)(5, 5, 5, 9, 6, 6)  # second box overlaps the first
    assert L.chemora_amr_create_boxes(N.BSSN, nc3, 2, ov_lo, two_hi, 0.1, None, ctypes.byref(a)) == N.EINVAL
    assert L.chemora_amr_create_boxes(N.WAVE_VARC, nc3, 2, two_lo, two_hi, 0.1, None, ctypes.byref(a)) == N.EINVAL
    assert L.chemora_amr_create_boxes(N.BSSN, nc3, 0, two_lo, two_hi, 0.1, None, ctypes.byref(a)) == N.EINVAL
    assert L.chemora_amr_step_mode(None, 0.1, 1, 0, None) == N.EINVAL
