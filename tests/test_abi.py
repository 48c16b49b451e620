"""The C ABI without a GPU: libhologen.so loads, exports every function that
include/hologen.h declares, and its host-only logic (defaults, size support,
status strings, argument checks made before any device work) behaves as the
header documents."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_12214_gb300 import build, hologen
    if not os.path.exists(build.LIB):
        build.build()
    return hologen.lib()


def declared_functions():
    src = "\n".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = "\n".join(l for l in src.splitlines() if not l.lstrip().startswith("#"))
    names = re.findall(r"\b(hg_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_documented_entry_points():
    names = declared_functions()
    for must in ("hg_plan_create", "hg_run", "hg_replay", "hg_debug_step", "hg_sync",
                 "hg_plan_destroy", "hg_group_run"):
        assert must in names
    for must in ("hg_cnn_create", "hg_cnn_train_step", "hg_conv3x3_forward", "hg_conv3x3_wgrad"):
        assert must in names
    assert len(names) >= 40


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults_and_status_strings(lib):
    from paper_2008_12214_gb300 import hologen as hg
    o = hg.hg_opts()
    lib.hg_opts_default(ctypes.byref(o))
    assert (o.subframes, o.use_graph, o.pipeline, o.autotune, o.precision, o.seed) == (24, 1, -1, 1, 0, 0)
    assert o.host_chunks == 0
    seen = set()
    for st in range(8):
        s = hg.hg_status_string(st)
        assert s and s != "unknown status"
        seen.add(s)
    assert len(seen) == 8
    assert hg.hg_status_string(99) == "unknown status"


def test_supported_lengths_are_2_3_5_smooth_and_compiled(lib):
    from paper_2008_12214_gb300 import hologen as hg
    for n in (4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 1080, 1920, 30, 60, 96):
        assert hg.hg_supported_length(n), n
    for n in (0, 1, 7, 14, 1000, 1023, 4096, -8):
        assert not hg.hg_supported_length(n), n


@pytest.mark.parametrize("ny,nx,batch,kind,levels,algo,want", [
    (64, 64, 0, 0, 2, 0, 1),       # batch < 1
    (0, 64, 1, 0, 2, 0, 1),        # ny < 1
    (64, 64, 1, 5, 2, 0, 1),       # unknown SLM kind
    (64, 64, 1, 1, 1, 0, 1),       # L-level with L < 2
    (64, 64, 1, 1, 257, 0, 1),     # L-level with L > 256
    (64, 64, 1, 1, 4, 2, 1),       # OSPR needs a binary SLM
    (64, 64, 1, 0, 2, 7, 1),       # unknown algorithm
    (64, 1000, 1, 0, 2, 0, 2),     # 1000 is not a compiled length
    (14, 64, 1, 0, 2, 0, 2),       # nor 14
])
def test_plan_create_rejects_bad_arguments_before_device_work(lib, ny, nx, batch, kind, levels, algo, want):
    from paper_2008_12214_gb300 import hologen as hg
    h = ctypes.c_void_p(123)
    st = lib.hg_plan_create(ctypes.byref(h), ny, nx, batch, hg.hg_slm(kind, levels), algo, None)
    assert st == want
    assert h.value is None


def test_null_handles_are_rejected(lib):
    assert lib.hg_run(None, None, None, 1, None, None) == 1
    assert lib.hg_sync(None) == 1
    assert lib.hg_replay(None, None, None) == 1
    assert lib.hg_last_launch_count(None) == 0
    lib.hg_plan_destroy(None)


def test_plain_c_client_builds_and_runs(tmp_path):
    """The boundary is a C ABI: a C program compiled with gcc against
    include/*.h alone, linked to libhologen.so, runs the calls that need no
    GPU."""
    import shutil
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2008_12214_gb300")
    if not os.path.exists(os.path.join(pkg, "libhologen.so")) or shutil.which("gcc") is None:
        pytest.skip("library or gcc missing")
    exe = str(tmp_path / "c_abi_check")
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                           os.path.join(root, "tests", "c_abi_check.c"), "-L", pkg, "-lhologen",
                           "-Wl,-rpath," + pkg, "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and "c abi ok" in out.stdout, (out.returncode, out.stdout, out.stderr)


@pytest.mark.parametrize("ny,nx,kind,levels,algo,opt,value,want", [
    (256, 256, 0, 2, 5, None, None, 2),        # direct search: 65536 pixels exceed one CTA's shared memory
    (32, 32, 0, 2, 6, "sa_temp", 0.0, 1),      # annealing needs a positive temperature
    (32, 32, 0, 2, 6, "sa_cool", 1.5, 1),      # and a cooling factor in (0, 1]
    (32, 32, 2, 4, 5, None, None, 1),          # search plans are phase-SLM plans
    (64, 64, 0, 2, 1, "modulated", 1, 1),      # modulated plans run GS only
    (64, 64, 0, 2, 0, "fresnel", float("nan"), 1),
    (64, 64, 2, 8, 0, "amp_clip", 0.0, 1),     # amplitude SLM needs a positive clip
    (64, 64, 2, 257, 0, None, None, 1),        # amplitude SLM with L > 256
    (1024, 1024, 0, 2, 0, "precision", 5, 1),  # precision outside 0..4
    (64, 64, 0, 2, 4, "lt_start", 0.0, 1),     # Liu-Taghizadeh window fraction in (0, 1]
    (64, 64, 0, 2, 0, "host_chunks", -1, 1),   # chunk count >= 0
])
def test_variant_options_rejected_before_device_work(lib, ny, nx, kind, levels, algo, opt, value, want):
    from paper_2008_12214_gb300 import hologen as hg
    o = hg.hg_opts()
    lib.hg_opts_default(ctypes.byref(o))
    if opt is not None:
        setattr(o, opt, value)
    if opt == "precision":
        o.modulated = 1
    h = ctypes.c_void_p(123)
    st = lib.hg_plan_create(ctypes.byref(h), ny, nx, 1, hg.hg_slm(kind, levels), algo, ctypes.byref(o))
    assert st == want, st
    assert h.value is None
