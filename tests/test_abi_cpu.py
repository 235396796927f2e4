"""CPU checks of the C ABI: the library builds, loads, exports every symbol
include/g6gb.h declares, and fails cleanly (no crash, an error code) where no
GPU exists.  No compute call runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_0902_4463_gb300 import build, g6gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "g6gb.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return g6gb.lib()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(g6[a-z0-9_]*)\s*\(", text))
    names -= {"g6x_alloc_fn", "g6x_free_fn"}
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 30
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(g6gb.EXPORTS)


def test_record_layouts_match_header():
    # g6x_jrec 120 B, g6x_irec 64 B, g6x_out 64 B as documented in g6gb.h
    assert g6gb.JREC.itemsize == 120
    assert g6gb.IREC.itemsize == 64
    assert g6gb.OUT.itemsize == 64


def test_paper_constants_golden(lib):
    # tests/golden/paper_constants.txt holds the numbers the paper prints
    vals = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_constants.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = int(v)
    assert g6gb.g6_npipes() == vals["npipes"]
    assert g6gb.G6_MAXNB == vals["max_neighbours"]
    from bench import FLOPS_PER_PAIR, FLOPS_PER_PAIR_DS
    assert FLOPS_PER_PAIR == vals["flops_per_pair"]
    assert FLOPS_PER_PAIR_DS == vals["flops_per_pair_ds"]
    assert vals["flops_per_pair_ds"] - vals["flops_per_pair"] == 3 * (vals["ds_sub_flops"] - 1)


def test_strerror_and_argument_errors_without_gpu(lib):
    assert g6gb.strerror(g6gb.G6_EINVAL) == "invalid argument"
    assert g6gb.strerror(g6gb.G6_EOVERFLOW) == "neighbour list overflow"
    assert lib.g6_open(-1) == g6gb.G6_EINVAL
    assert lib.g6_open(g6gb.G6_MAX_CLUSTERS) == g6gb.G6_EINVAL
    assert lib.g6_close(3) == g6gb.G6_ENOTOPEN
    assert lib.g6_set_ti(3, 0.0) == g6gb.G6_ENOTOPEN
    assert lib.g6x_set_precision(3, 0) == g6gb.G6_ENOTOPEN
    assert lib.g6_set_tunit(51) == 0 and lib.g6_set_xunit(51) == 0


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="host has a GPU")
def test_open_without_gpu_reports_enodev(lib):
    assert lib.g6_open(0) == g6gb.G6_ENODEV
    assert lib.g6x_open_ex(1, 1024, 256) == g6gb.G6_ENODEV
    err = ctypes.c_int(0)
    nj = (ctypes.c_int * 2)(300, 17)
    assert not lib.g6x_batch_create(2, nj, 0, 0, 0, ctypes.byref(err))
    assert err.value == g6gb.G6_ENODEV


def test_batch_argument_checks_need_no_gpu(lib):
    err = ctypes.c_int(0)
    nj = (ctypes.c_int * 2)(300, 17)
    assert not lib.g6x_batch_create(0, nj, 0, 0, 0, ctypes.byref(err))
    assert err.value == g6gb.G6_EINVAL
    assert not lib.g6x_batch_create(2, nj, 1, 0, 0, ctypes.byref(err))   # FP64: not batched
    assert err.value == g6gb.G6_EINVAL
    assert not lib.g6x_batch_create(2, nj, 0, 99, 0, ctypes.byref(err))
    assert err.value == g6gb.G6_EINVAL
    assert lib.g6x_batch_calc(None, None, None, None, 0) == g6gb.G6_EINVAL
    assert lib.g6x_batch_destroy(None) == g6gb.G6_EINVAL
    assert lib.g6hb_step(None, 1.0) == g6gb.G6_EINVAL
    assert lib.g6x_batch_launch_count(None) == 0


def test_binding_refuses_missing_library(tmp_path, monkeypatch):
    monkeypatch.setattr(g6gb, "_lib", None)
    monkeypatch.setattr(g6gb, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        g6gb.lib()


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_0902_4463_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle.h" not in text and "liboracle" not in text, f


def test_tuning_table_file_round_trip(lib, tmp_path):
    p = tmp_path / "tune.txt"
    p.write_text("# table\n0 4 4 1\n0 5 3 2\n0 17 0 1\n1 10 7 1\n")
    assert g6gb.g6x_load_tuning(p) == 4
    bad = tmp_path / "bad.txt"
    bad.write_text("0 4 99 1\n")                  # unknown variant
    with pytest.raises(g6gb.G6Error):
        g6gb.g6x_load_tuning(bad)
    bad.write_text("1 4 0 1\n")                   # DS variant under FP64
    with pytest.raises(g6gb.G6Error):
        g6gb.g6x_load_tuning(bad)
    assert g6gb.g6x_clear_tuning() == 0


def test_wait_limit_range(lib):
    assert lib.g6x_set_wait_limit(0.0) == g6gb.G6_EINVAL
    assert lib.g6x_set_wait_limit(1e-7) == g6gb.G6_EINVAL
    assert lib.g6x_set_wait_limit(3.0) == g6gb.G6_EINVAL
    assert lib.g6x_set_wait_limit(float("nan")) == g6gb.G6_EINVAL
    assert lib.g6x_set_wait_limit(0.5) == 0
    assert lib.g6x_set_wait_limit(2.0) == 0
    assert lib.g6x_probe_wait_timeout(9) == g6gb.G6_ENOTOPEN


def _build_c_client(tmp_path):
    """Compile and link the plain-C GRAPE client against the header and the
    library (the library's directory as its run path)."""
    import subprocess
    libdir = os.path.join(ROOT, "paper_0902_4463_gb300")
    exe = str(tmp_path / "grape_client")
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-O1",
           os.path.join(ROOT, "tests", "c_client", "grape_client.c"),
           "-I", os.path.join(ROOT, "include"), "-L", libdir, "-lg6gb",
           "-Wl,-rpath," + libdir, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_builds_against_the_header_and_library(lib, tmp_path):
    import subprocess
    exe = _build_c_client(tmp_path)
    inp = tmp_path / "in.txt"
    inp.write_text("2\n0.5 0 0 0 0 0 0\n0.5 1 0 0 0 0 0\n")
    r = subprocess.run([exe, str(inp), str(tmp_path / "out.txt"), "1e-4", "0"],
                       capture_output=True, text=True)
    if not os.path.exists("/dev/nvidia0"):
        assert r.returncode == -g6gb.G6_ENODEV          # no GPU here


def test_launch_plan_heuristic_without_a_gpu(lib):
    """The built-in launch choice (g6x_plan_launch, no GPU needed): the
    widest i-tile that the block size allows, narrowed while the work line
    holds too few (i-tile, j-tile) units -- the shapes the autotuner measured
    best at N = 2^20 and at N = 32768."""
    g6gb.g6x_clear_tuning()
    ds = g6gb.G6X_PREC_DS

    def shape(nj, ni, mode=ds, list_=False):
        p = g6gb.g6x_plan_launch(mode, nj, ni, list_)
        assert p["jtiles"] == (nj + 255) // 256
        assert 1 <= p["grid"] <= -(-ni // (p["ti"] * p["ni_per"])) * p["jtiles"]
        return p["ti"], p["tj"], p["ni_per"]

    big, small = 1 << 20, 32768

    def ws(nj, ni):
        return g6gb.g6x_variant_info(g6gb.g6x_plan_launch(ds, nj, ni)["variant"])["ws"] == 1

    # blocks of up to 16 take the small-block kernel with the narrowest
    # i-tile that holds them, blocks of up to 32 too from 512 j-tiles on,
    # blocks of up to 64 from 2048 j-tiles on; larger blocks the split-j
    # and wide shapes
    for nj in (1024, small, 131072, 524288, big):
        assert all(ws(nj, ni) for ni in (1, 8, 9, 16))
        assert all(ws(nj, ni) == (nj >= 131072) for ni in (17, 32))
        assert all(ws(nj, ni) == (nj >= 524288) for ni in (33, 64))
        assert not any(ws(nj, ni) for ni in (65, 128, 256, 4096))
        assert shape(nj, 1) == (8, 32, 1) and shape(nj, 8) == (8, 32, 1)
        lp = g6gb.g6x_plan_launch(ds, nj, 16, True)                      # lists: no
        assert g6gb.g6x_variant_info(lp["variant"])["ws"] == 0
        assert g6gb.g6x_variant_info(lp["variant"])["list"] == 1
    assert shape(big, 17) == (32, 8, 1) and shape(big, 64) == (64, 4, 1)
    assert shape(big, 16) == (16, 16, 1)
    assert shape(big, 128) == (32, 8, 2)
    assert shape(big, 256) == (64, 4, 2)
    assert shape(big, 2048) == (64, 4, 2)
    assert shape(big, 4096) == (128, 1, 2)
    assert shape(big, big) == (128, 1, 2)
    # the widest tiles run 4 CTAs per SM (the occupancy query needs a GPU:
    # one without), in more waves on longer work lines
    for ni, waves in ((4096, 1), (16384, 2), (65536, 2), (262144, 4), (big, 8)):
        p = g6gb.g6x_plan_launch(ds, big, ni)
        assert p["variant"] == 9 and p["grid"] in (152 * waves, 152 * 4 * waves), (ni, p)
    assert shape(small, 256) == (16, 16, 1)
    assert shape(small, 1024) == (32, 8, 2)
    assert shape(small, 4096) == (64, 4, 2)
    assert shape(small, small) == (64, 4, 2)        # 16384 units: below the wide tile's 65536
    assert shape(131072, 16384) == (64, 4, 2) and shape(131072, 65536) == (128, 1, 2)
    # a smaller j-set never gets a wider i-tile at the same block size
    for ni in (16, 64, 200, 1000, 3000, 20000):
        widths = [np.prod(shape(nj, ni)[::2]) for nj in (4096, 32768, 131072, 1 << 20)]
        assert widths == sorted(widths), (ni, widths)
    # other modes keep their own kernels
    assert g6gb.g6x_plan_launch(g6gb.G6X_PREC_FP64, big, 4096)["variant"] == 7
    assert g6gb.g6x_plan_launch(g6gb.G6X_PREC_FP64, big, 4096, True)["variant"] == 8
    # lists take the twins of the three-kernel path's shapes, the widest
    # only from 2^18 (i-tile, j-tile) units on
    for nj in (small, 131072, big):
        for ni in (16, 32, 64, 128, 256, 1000, 4096, 20000, nj):
            lp = g6gb.g6x_plan_launch(ds, nj, ni, True)
            info = g6gb.g6x_variant_info(lp["variant"])
            assert info["list"] == 1 and info["prec"] == ds and info["ws"] == 0
            if ni > 64:
                wl, wp = shape(nj, ni, ds, True), shape(nj, ni)
                assert wl == wp or (wp == (128, 1, 2) and wl == (64, 4, 2)), (nj, ni)
                assert (wl == (128, 1, 2)) == (-(-ni // 256) * (nj // 256) >= 1 << 18), (nj, ni)
    assert shape(big, 16, ds, True) == (16, 16, 1)
    assert shape(131072, 16384, ds, True) == (64, 4, 2)
    assert shape(big, 4096, ds, True) == (64, 4, 2)
    assert shape(big, 65536, ds, True) == (128, 1, 2)
    assert g6gb.g6x_plan_launch(g6gb.G6X_PREC_DS_DSSUB, big, 16)["variant"] == 22
    assert g6gb.g6x_plan_launch(g6gb.G6X_PREC_DS_DSSUB, big, 4096)["variant"] == 21
    out = np.zeros(6, dtype=np.int32)
    p = out.ctypes.data_as(ctypes.c_void_p)
    for args in ((9, big, 16, 0, 152), (ds, 0, 16, 0, 152), (ds, big, 0, 0, 152),
                 (ds, big, 16, 0, 0), (g6gb.G6X_PREC_DS_DSSUB, big, 16, 1, 152)):
        assert lib.g6x_plan_launch(*args, p) == g6gb.G6_EINVAL
    assert lib.g6x_plan_launch(ds, big, 16, 0, 152, None) == g6gb.G6_EINVAL


def test_tuning_table_is_consulted_and_loads_all_or_nothing(lib, tmp_path):
    """A table in the autotuner's format ("precision log2(m) variant
    grid_multiplier") overrides the built-in launch choice for its block-size
    buckets (larger buckets reuse the largest tuned one); the fused-prediction
    shapes only where the predictor allows them; a file with one bad line
    changes nothing; clearing restores the built-in choice."""
    ds, x64 = g6gb.G6X_PREC_DS, g6gb.G6X_PREC_DS_X64
    big = 1 << 20
    g6gb.g6x_clear_tuning()
    ws16 = g6gb.g6x_plan_launch(ds, big, 16)["variant"]      # the small-block kernel
    assert g6gb.g6x_variant_info(ws16)["ws"] == 1
    assert g6gb.g6x_plan_launch(x64, big, 16)["variant"] == 4   # no fused prediction there
    good = tmp_path / "good.txt"
    good.write_text("# comment\n0 4 17 1\n0 5 14 2\n1 4 7 1\n")
    assert g6gb.g6x_load_tuning(str(good)) == 3
    assert g6gb.g6x_plan_launch(ds, big, 16)["variant"] == 17
    assert g6gb.g6x_plan_launch(x64, big, 16)["variant"] == 4      # its separate twin
    p32 = g6gb.g6x_plan_launch(ds, big, 32)
    assert p32["variant"] == 14
    assert g6gb.g6x_plan_launch(ds, big, 4096)["variant"] == 14    # largest bucket reused
    assert g6gb.g6x_plan_launch(g6gb.G6X_PREC_FP64, big, 16)["variant"] == 7
    for bad in ("0 4 99 1\n", "0 4 7 1\n", "0 4 5 1\n", "0 4 4 9\n", "2 4 4 1\n", "0 4\n"):
        f = tmp_path / "bad.txt"
        f.write_text("0 6 16 1\n" + bad)
        with np.testing.assert_raises(g6gb.G6Error):
            g6gb.g6x_load_tuning(str(f))
        assert g6gb.g6x_plan_launch(ds, big, 64)["variant"] == 14, bad   # nothing applied
    with np.testing.assert_raises(g6gb.G6Error):
        g6gb.g6x_load_tuning(str(tmp_path / "missing.txt"))
    g6gb.g6x_clear_tuning()
    assert g6gb.g6x_plan_launch(ds, big, 16)["variant"] == ws16
    assert g6gb.g6x_plan_launch(ds, big, 4096)["variant"] == 9


def test_driver_setters_refuse_bad_arguments_without_a_gpu(lib):
    """The drivers' option setters validate before touching any state: a NULL
    driver handle is refused, as is a force-noise allowance outside [0, 1)
    in the stand-alone corrector."""
    assert lib.g6h_set_force_noise(None, 0.1) == g6gb.G6_EINVAL
    assert lib.g6hb_set_force_noise(None, 0.1) == g6gb.G6_EINVAL
    assert lib.g6h_set_neighbour_radius(None, 1e-4) == g6gb.G6_EINVAL
    z = np.zeros((1, 3))
    for bad in (-1e-9, float("nan")):
        with pytest.raises(g6gb.G6Error):
            g6gb.g6h_correct_block(0.5, [0.25], [0.25], 0.01, 0.5, 2.0 ** -40, z, z, z, z, z, z,
                                   force_noise=bad)
