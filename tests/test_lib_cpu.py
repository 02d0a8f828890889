"""The C-ABI library builds, loads and exports every symbol of include/ftgemm.h;
host-only logic (argument codes, injection settings, error strings) works
without a GPU.  No compute call is made here."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ft():
    from paper_2305_02444_gb300 import build
    build.build()
    from paper_2305_02444_gb300 import ftgemm
    ftgemm.lib()
    return ftgemm


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+(ftgemm_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ftgemm_d", "ftgemm_d_noft", "ftgemm_d_host", "ftgemm_encode_operands",
                 "ftgemm_set_injection", "ftgemm_injection_log", "ftgemm_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(ft):
    """Exactly the functions the header declares: the internal launchers and
    library templates stay local (linker version script)."""
    out = subprocess.run(["nm", "-D", "--defined-only", ft.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(l.split()[-1].split("@")[0] for l in out.splitlines() if l.strip())
    exported.discard("")
    for name in declared_functions():
        assert name in exported, name
        assert getattr(ft.lib(), name) is not None
    assert exported == set(declared_functions()), sorted(exported ^ set(declared_functions()))


def test_build_targets_sm103a_only():
    from paper_2305_02444_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.parametrize("args,code", [
    (("X", "N", 2, 2, 2, 2, 2, 2), -1), (("N", "Q", 2, 2, 2, 2, 2, 2), -2),
    (("N", "N", -1, 2, 2, 2, 2, 2), -3), (("N", "N", 2, -1, 2, 2, 2, 2), -4),
    (("N", "N", 2, 2, -1, 2, 2, 2), -5), (("N", "N", 3, 2, 2, 2, 2, 3), -8),
    (("T", "N", 2, 2, 3, 2, 3, 2), -8), (("N", "N", 2, 2, 3, 2, 2, 2), -10),
    (("N", "T", 2, 3, 2, 2, 2, 2), -10), (("N", "N", 3, 2, 2, 3, 2, 2), -13),
])
def test_argument_codes_without_device(ft, args, code):
    ta, tb, M, N, K, lda, ldb, ldc = args
    assert ft.ftgemm_d(ta, tb, M, N, K, 1.0, 0, lda, 0, ldb, 0.0, 0, ldc, report=False, stream=0)[0] == code
    assert ft.ftgemm_d_noft(ta, tb, M, N, K, 1.0, 0, lda, 0, ldb, 0.0, 0, ldc, stream=0) == code
    assert ft.ftgemm_d_host(ta, tb, M, N, K, 1.0, 0, lda, 0, ldb, 0.0, 0, ldc, stream=0)[0] == code


def test_split_slice_count_checked_without_device(ft):
    assert ft.ftgemm_d_split("N", "N", 4, 4, 4, 1.0, 0, 4, 0, 4, 0.0, 0, 4, nslices=16, report=False, stream=0)[0] == -14
    assert ft.ftgemm_d_split("N", "N", 4, 4, 4, 1.0, 0, 4, 0, 4, 0.0, 0, 4, nslices=-1, report=False, stream=0)[0] == -14


def test_host_settings_and_strings(ft):
    assert ft.ftgemm_set_injection(mode=0) == 0
    assert ft.ftgemm_set_injection(mode=1, seed=5, count=-1) == -1
    assert ft.ftgemm_set_injection(mode=7) == -1
    assert ft.ftgemm_set_injection(mode=2, flips=[(0, 0, 0, 3)]) == 0
    assert ft.ftgemm_set_injection(mode=0) == 0
    assert "timeout" in ft.ftgemm_strerror(ft.ERR_TIMEOUT) or "wait" in ft.ftgemm_strerror(ft.ERR_TIMEOUT)
    assert ft.ftgemm_strerror(0) == "success"
    assert ft.ftgemm_launch_count() == 0


def test_split_engine_knob_codes(ft):
    for e in (8, 6, 4, 3, -1):   # 3, 4 and 6 (cluster forms) no longer exist
        assert ft.ftgemm_set_split_engine(e) == -1
    for e in (7, 5, 2):
        assert ft.ftgemm_set_split_engine(e) == 0
    assert ft.ftgemm_set_split_engine(1) == 0
    assert ft.ftgemm_set_split_engine(0) == 0


def test_host_panels_knob_codes(ft):
    assert ft.ftgemm_set_host_panels(-1) == -1
    for n in (3, 1, 0):
        assert ft.ftgemm_set_host_panels(n) == 0


def test_correction_knob_codes(ft):
    assert ft.ftgemm_set_correction(2) == -1
    assert ft.ftgemm_set_correction(-1) == -1
    assert ft.ftgemm_set_correction(1) == 0
    assert ft.ftgemm_set_correction(0) == 0


def test_autotune_signature_and_cache(tmp_path, monkeypatch):
    """The batched schedule autotuner's host side: the batch signature is the
    multiset of (layouts, shape) -- order-free, sensitive to every field --,
    a missing or corrupt cache reads as empty, and a cached signature returns
    its schedule without timing anything."""
    import json
    from paper_2305_02444_gb300 import autotune
    monkeypatch.setattr(autotune, "_device_name", lambda: "cpu")
    shapes = [("N", "N", 100, 200, 300), ("T", "N", 64, 64, 64), ("N", "T", 1024, 32, 77)]
    sig = autotune.signature(shapes)
    assert sig == autotune.signature(list(reversed(shapes)))
    for k in range(5):
        changed = [list(s) for s in shapes]
        changed[0][k] = "T" if k < 2 else changed[0][k] + 1
        assert autotune.signature([tuple(s) for s in changed]) != sig
    assert len(set(autotune.CANDIDATES)) == len(autotune.CANDIDATES) == 9
    path = tmp_path / "sched.json"
    assert autotune.load_cache(str(path)) == {}
    path.write_text("{not json")
    assert autotune.load_cache(str(path)) == {}
    path.write_text(json.dumps({f"cpu:{sig}": {"schedule": 17, "ms": {"17": 1.0}, "n": 3}}))
    best, ms = autotune.tune_batched(shapes, cache_path=str(path))
    assert best == 17 and ms == {"17": 1.0}


@pytest.mark.parametrize("call", ["d", "noft", "host", "noalloc", "unfused", "split"])
def test_empty_output_returns_before_the_device(ft, call):
    """M = 0 or N = 0: nothing to compute, 0 returned before any device work."""
    for M, N in ((0, 3), (3, 0)):
        args = ("N", "N", M, N, 4, 1.0, 0, max(1, M), 0, 4, 0.5, 0, max(1, M))
        if call == "d":
            rc = ft.ftgemm_d(*args, stream=0)[0]
        elif call == "noft":
            rc = ft.ftgemm_d_noft(*args, stream=0)
        elif call == "host":
            rc = ft.ftgemm_d_host(*args, stream=0)[0]
        elif call == "noalloc":
            rc = ft.ftgemm_d_noalloc(*args, stream=0)[0]
        elif call == "unfused":
            rc = ft.ftgemm_d_unfused(*args, stream=0)[0]
        else:
            rc = ft.ftgemm_d_split(*args, nslices=7, ft=2, stream=0)[0]
        assert rc == 0, (call, M, N, rc)
    assert ft.ftgemm_launch_count() == 0


@pytest.mark.parametrize("args,code", [
    (("X", "N", 2, 2, 2, 2, 2, 2), -1), (("N", "N", -1, 2, 2, 2, 2, 2), -3),
    (("N", "N", 3, 2, 2, 2, 2, 3), -8), (("N", "T", 2, 3, 2, 2, 2, 2), -10),
    (("N", "N", 3, 2, 2, 3, 2, 2), -13),
])
def test_other_entry_points_number_arguments_as_ftgemm_d(ft, args, code):
    ta, tb, M, N, K, lda, ldb, ldc = args
    full = (ta, tb, M, N, K, 1.0, 0, lda, 0, ldb, 0.0, 0, ldc)
    assert ft.ftgemm_d_noalloc(*full, report=False, stream=0)[0] == code
    assert ft.ftgemm_d_unfused(*full, report=False, stream=0)[0] == code
    assert ft.ftgemm_d_split(*full, nslices=3, ft=2, report=False, stream=0)[0] == code


def test_split_checksum_form_code(ft):
    base = ("N", "N", 4, 4, 4, 1.0, 0, 4, 0, 4, 0.0, 0, 4)
    for nslices, ftflag in ((3, 3), (3, -1), (0, 2)):   # ft 2 needs an emulated form
        assert ft.ftgemm_d_split(*base, nslices=nslices, ft=ftflag, report=False, stream=0)[0] == -15


@pytest.mark.parametrize("args,code", [
    (("X", "N", 2, 2, 2, 2, 2), -1), (("N", "Q", 2, 2, 2, 2, 2), -2), (("N", "N", -1, 2, 2, 2, 2), -3),
    (("N", "N", 2, -1, 2, 2, 2), -4), (("N", "N", 2, 2, -1, 2, 2), -5), (("N", "N", 3, 2, 2, 2, 2), -7),
    (("T", "N", 2, 2, 3, 2, 3), -7), (("N", "N", 2, 2, 3, 2, 2), -9), (("N", "T", 2, 3, 2, 2, 2), -9),
    (("N", "N", 0, 2, 2, 1, 2), 0), (("N", "N", 2, 2, 0, 2, 1), 0),
])
def test_encode_operands_argument_codes(ft, args, code):
    """ftgemm_encode_operands numbers its own arguments (lda 7, ldb 9); an
    empty problem returns 0 before the device."""
    ta, tb, M, N, K, lda, ldb = args
    z = [0] * 6
    assert ft.ftgemm_encode_operands(ta, tb, M, N, K, 0, lda, 0, ldb, *z, stream=0) == code


def test_batched_argument_codes_before_the_device(ft):
    """-(100 p + i) for argument i (ftgemm_d's numbering) of problem p; count
    < 0, a NULL per-problem array or a NULL plan pointer: FTGEMM_ERR_BATCH;
    the plan calls on a NULL plan: -1.  All found before any device work."""
    import ctypes
    L = ft.lib()
    ok = ("N", "N", 4, 4, 4, 1.0, 0, 4, 0, 4, 0.0, 0, 4)
    assert ft.ftgemm_batched([ok, ("N", "N", 4, 4, 4, 1.0, 0, 3, 0, 4, 0.0, 0, 4)])[0] == -108
    assert ft.ftgemm_batched([("N", "Z") + ok[2:], ok])[0] == -2
    assert ft.ftgemm_batched([ok, ok, ("N", "N", 4, 4, 4, 1.0, 0, 4, 0, 4, 0.0, 0, 3)])[0] == -213
    a = ft._BatchArgs([ok])
    args = list(a.args())
    assert L.ftgemm_batched(-1, *args[1:], None, None) == ft.ERR_BATCH
    for k in range(1, len(args)):
        nulled = list(args)
        nulled[k] = None
        assert L.ftgemm_batched(1, *nulled[1:], None, None) == ft.ERR_BATCH, k
    assert L.ftgemm_batched_plan_create(None, *args, 1, -1, None) == ft.ERR_BATCH
    h = ctypes.c_void_p()
    assert L.ftgemm_batched_plan_create(ctypes.byref(h), -3, *args[1:], 1, -1, None) == ft.ERR_BATCH
    assert not h.value
    assert L.ftgemm_batched_plan_launch(None, None) == -1
    assert L.ftgemm_batched_plan_report(None, None, None) == -1
    assert L.ftgemm_batched_plan_injection_log(None, None, 0) == -1
    assert L.ftgemm_batched_plan_destroy(None) == -1
    assert "batch" in ft.ftgemm_strerror(ft.ERR_BATCH)
    assert ft.ftgemm_launch_count() == 0


def test_ksplit_plan_of_the_measured_shapes(ft):
    """On 152 SMs: 1024^3 (64 tiles) splits every tile; 4096^3 (1024 tiles,
    6 waves + 112) runs 912 tiles whole and splits the 112 tail tiles 4 ways;
    8192^3 (4096 tiles, the last wave 144 of 152) and the rank-256 update do
    not split."""
    assert ft.ftgemm_query_ksplit(4096, 4096, 4096) == (0, 4, 912)
    rc, S, first = ft.ftgemm_query_ksplit(1024, 1024, 1024)
    assert rc == 0 and S > 1 and first == 0
    assert ft.ftgemm_query_ksplit(8192, 8192, 8192) == (0, 1, 4096)
    assert ft.ftgemm_query_ksplit(8192, 8192, 256) == (0, 1, 4096)


def test_ksplit_plan_properties(ft):
    """For any shape: 1 <= S <= 32 k-ranges, none empty; S = 1 exactly when no
    tile is split; grids under 4 tiles per SM split all tiles or none; larger
    grids split at most their last, partly empty wave."""
    import random
    rng = random.Random(4)
    for nsm in (152, 148, 7):
        for _ in range(400):
            M, N = rng.randint(1, 12000), rng.randint(1, 12000)
            K = rng.choice([rng.randint(1, 64), rng.randint(1, 40000)])
            rc, S, first = ft.ftgemm_query_ksplit(M, N, K, nsm)
            assert rc == 0
            ntiles = -(-M // 128) * -(-N // 128)
            nks = -(-K // 16)
            assert 1 <= S <= min(32, nks)
            ks = -(-nks // S)
            assert -(-nks // ks) == S                    # S non-empty k-ranges
            assert (S == 1) == (first == ntiles)
            if ntiles < 4 * nsm:
                assert first in (0, ntiles)
            else:
                assert first in (ntiles - ntiles % nsm, ntiles)
                assert S == 1 or ntiles % nsm != 0


def test_ksplit_plan_follows_the_knobs(ft):
    try:
        assert ft.ftgemm_set_splitk(1) == 0
        for n in (256, 1024, 4096):
            assert ft.ftgemm_query_ksplit(n, n, n) == (0, 1, (n // 128) ** 2)
        assert ft.ftgemm_set_splitk(4) == 0
        assert ft.ftgemm_query_ksplit(1024, 1024, 1024) == (0, 4, 0)
        assert ft.ftgemm_query_ksplit(4096, 4096, 4096) == (0, 4, 0)   # forced: every tile
        assert ft.ftgemm_query_ksplit(256, 256, 32) == (0, 2, 0)       # 2 k-slabs: 2 splits
        assert ft.ftgemm_set_splitk(0) == 0
        assert ft.ftgemm_set_panel_check(16) == 0
        # panel checks run inside the k-splits: the plan is the same with or without them
        assert ft.ftgemm_query_ksplit(1024, 1024, 1024)[1] > 1
        assert ft.ftgemm_query_ksplit(1024, 1024, 160)[1] > 1
    finally:
        ft.ftgemm_set_splitk(0)
        ft.ftgemm_set_panel_check(0)


def test_ksplit_query_arguments(ft):
    import ctypes
    L = ft.lib()
    sp, first = ctypes.c_int(0), ctypes.c_int64(0)
    for args, code in (((-1, 4, 4, 152), -1), ((4, -1, 4, 152), -2), ((4, 4, -1, 152), -3),
                       ((4, 4, 4, 0), -4)):
        assert L.ftgemm_query_ksplit(*args, ctypes.byref(sp), ctypes.byref(first)) == code
    assert L.ftgemm_query_ksplit(4, 4, 4, 152, None, ctypes.byref(first)) == -5
    assert L.ftgemm_query_ksplit(4, 4, 4, 152, ctypes.byref(sp), None) == -6
    assert ft.ftgemm_query_ksplit(0, 300, 300) == (0, 1, 0)
    assert ft.ftgemm_query_ksplit(300, 300, 0) == (0, 1, 9)


def test_binding_refuses_addresses_a_kernel_cannot_use(ft):
    """Device arguments take CUDA float64 tensors or raw pointers; host
    arguments (ftgemm_d_host) CPU float64 tensors or numpy arrays.  A tensor
    on the wrong side or of another dtype raises before the library is called."""
    import numpy as np
    import torch

    class CudaLike:   # what the binding reads from a CUDA tensor
        is_cuda = True
        dtype = torch.float64
        device = "cuda:0"

        def data_ptr(self):
            return 4096

    cpu64 = torch.zeros(16, dtype=torch.float64)
    arr = np.zeros(16)
    assert ft._ptr(CudaLike()) == 4096
    assert ft._ptr(cpu64, device=False) == cpu64.data_ptr()
    assert ft._ptr(arr, device=False) == arr.ctypes.data
    assert ft._ptr(None) is None and ft._ptr(77) == 77
    for bad, device in ((cpu64, True), (arr, True), (CudaLike(), False),
                        (torch.zeros(4, dtype=torch.float32), False), (np.zeros(4, np.float32), False)):
        with pytest.raises(ValueError):
            ft._ptr(bad, device=device)
    with pytest.raises(TypeError):
        ft._ptr("not a buffer")
    with pytest.raises(ValueError):
        ft.ftgemm_d("N", "N", 4, 4, 4, 1.0, cpu64, 4, cpu64, 4, 0.0, cpu64, 4)
    with pytest.raises(ValueError):
        ft.ftgemm_d_host("N", "N", 4, 4, 4, 1.0, CudaLike(), 4, cpu64, 4, 0.0, cpu64, 4)
    assert ft.ftgemm_launch_count() == 0


def test_missing_library_raises(monkeypatch):
    """No fallback: without libftgemm.so every call raises."""
    from paper_2305_02444_gb300 import ftgemm
    monkeypatch.setattr(ftgemm, "_lib", None)
    monkeypatch.setattr(ftgemm, "LIB_PATH", os.path.join(ROOT, "_no_such_dir", "libftgemm.so"))
    with pytest.raises(RuntimeError):
        ftgemm.lib()
    with pytest.raises(RuntimeError):
        ftgemm.ftgemm_d("N", "N", 4, 4, 4, 1.0, 0, 4, 0, 4, 0.0, 0, 4)


def test_product_code_never_imports_the_oracle():
    """The package (the product path) has no import of the oracle, and no
    committed Python file reaches into the scratch folder.  bench.py imports
    the oracle only in oracle_sample (the CPU baseline and the reference arm),
    in flip_accounting (the CPU leg's classification of one call's faults,
    after the timed regions) and in the optional --split / --config5 /
    --panel-sweep reports,
    which check sampled rows outside their timed regions."""
    import ast
    pkg = os.path.join(ROOT, "paper_2305_02444_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(dirpath, f)).read()
                for node in ast.walk(ast.parse(src)):
                    if isinstance(node, ast.Import):
                        assert not any(a.name.split(".")[0] == "oracle" for a in node.names), f
                    elif isinstance(node, ast.ImportFrom):
                        assert (node.module or "").split(".")[0] != "oracle", f
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    allowed = {"oracle_sample", "flip_accounting", "split", "config5", "panel_sweep"}
    for fn in tree.body:
        for node in ast.walk(fn):
            names = ([a.name for a in node.names] if isinstance(node, ast.Import)
                     else [node.module or ""] if isinstance(node, ast.ImportFrom) else [])
            if any(n.split(".")[0] == "oracle" for n in names):
                assert isinstance(fn, ast.FunctionDef) and fn.name in allowed, getattr(fn, "name", "module level")
    scratch = re.compile(r"(?<![A-Za-z0-9_])" + "_" + r"work(?![A-Za-z0-9_])")   # the git-ignored scratch folder
    tracked = subprocess.run(["git", "ls-files", "*.py"], cwd=ROOT, capture_output=True, text=True).stdout.split()
    for f in tracked:
        if os.path.abspath(os.path.join(ROOT, f)) != os.path.abspath(__file__):
            assert not scratch.search(open(os.path.join(ROOT, f)).read()), f


def test_split_shape_limit_before_the_device(ft):
    """ftgemm_d_split refuses M or N above FTGEMM_SPLIT_MAX_ROWS (the slicing
    grids' limit) before any device work; at the limit it goes on (and, with
    no GPU here, stops at the device)."""
    big = ft.SPLIT_MAX_ROWS + 1
    assert ft.ftgemm_d_split("N", "N", big, 4, 4, 1.0, 0, big, 0, 4, 0.0, 0, big, nslices=3, ft=0,
                             report=False, stream=0)[0] == ft.ERR_TOO_LARGE
    assert ft.ftgemm_d_split("N", "N", 4, big, 4, 1.0, 0, 4, 0, 4, 0.0, 0, 4, nslices=0, ft=0,
                             report=False, stream=0)[0] == ft.ERR_TOO_LARGE
    at = ft.SPLIT_MAX_ROWS
    rc = ft.ftgemm_d_split("N", "N", at, 4, 4, 1.0, 0, at, 0, 4, 0.0, 0, at, nslices=3, ft=0,
                           report=False, stream=0)[0]
    assert rc != ft.ERR_TOO_LARGE
    assert "FTGEMM_SPLIT_MAX_ROWS" in ft.ftgemm_strerror(ft.ERR_TOO_LARGE)
    # K = 0: no slicing, the BLAS quick return applies at any size
    assert ft.ftgemm_d_split("N", "N", big, 4, 0, 1.0, 0, big, 0, 1, 1.0, 0, big, nslices=3, ft=0,
                             report=False, stream=0)[0] != ft.ERR_TOO_LARGE


def test_header_is_plain_c_and_a_c_caller_links(ft, tmp_path):
    """include/ftgemm.h compiles as C11 with warnings as errors (no C++ or
    torch types at the boundary); a C program links against libftgemm.so and
    runs the host-only paths without a GPU."""
    src = os.path.join(ROOT, "tests", "abi", "c_caller.c")
    exe = str(tmp_path / "c_caller")
    libdir = os.path.dirname(ft.LIB_PATH)
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"), src,
           "-o", exe, "-L", libdir, "-lftgemm", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr


def test_binding_structs_match_the_header_layout(ft, tmp_path):
    """Every struct of include/ftgemm.h has the same size and field offsets
    in C (compiled here) and in the binding's ctypes declarations."""
    exe = str(tmp_path / "layout")
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "abi", "layout.c"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    c_layout = dict(line.rsplit(" ", 1) for line in subprocess.run([exe], capture_output=True, text=True,
                                                                     check=True).stdout.splitlines())
    pairs = {"ftgemm_loc": ft.Loc, "ftgemm_report": ft.Report, "ftgemm_flip": ft.Flip,
             "ftgemm_inject": ft.Inject, "ftgemm_flip_log": ft.FlipLog}
    for cname, cls in pairs.items():
        assert int(c_layout[f"{cname} sizeof"]) == ctypes.sizeof(cls), cname
        c_fields = [k.split(".", 1)[1] for k in c_layout if k.startswith(cname + ".")]
        assert c_fields == [f for f, _ in cls._fields_], cname
        for f, _ in cls._fields_:
            assert int(c_layout[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_gpu_probes_compile():
    """The probe programs of the GPU tests include the kernel headers: they
    must keep compiling for sm_103a as those headers change (compiled here,
    run only on the GPU)."""
    import tempfile
    from paper_2305_02444_gb300 import build
    pdir = os.path.join(ROOT, "tests", "probes")
    with tempfile.TemporaryDirectory() as tmp:
        procs = []
        for f in sorted(os.listdir(pdir)):
            if f.endswith(".cu"):
                cmd = [build.nvcc()] + build.ARCH + ["-O3", "-std=c++17", "-I" + build.CSRC,
                                                     "-I" + os.path.join(ROOT, "include"), "-c",
                                                     os.path.join(pdir, f), "-o", os.path.join(tmp, f + ".o")]
                procs.append((f, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        assert procs
        for f, p in procs:
            out, _ = p.communicate(timeout=600)
            assert p.returncode == 0, (f, out.decode(errors="replace")[-2000:])
