"""The C ABI from plain C: tests/c_abi/client.c compiles as C11 with warnings
as errors against include/*.h alone, links to the built librearr.so, and its
host-only calls return what the Python binding sees."""
import os
import shutil
import subprocess

import pytest

from paper_1011_3583_gb300 import build as rbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    rbuild.build()
    from paper_1011_3583_gb300 import librearr
    libdir = os.path.dirname(librearr.lib_path())
    exe = str(tmp_path_factory.mktemp("c_abi") / "client")
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi", "client.c"), "-o", exe, "-L", libdir, "-lrearr",
           "-Wl,-rpath," + libdir]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    # the client reads the same tuning table as the Python binding
    env = dict(os.environ, REARR_TUNE_TABLE=librearr.DEFAULT_TUNE_TABLE)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, env=env).stdout
    return {ln.split()[0]: ln.split()[1:] for ln in out.splitlines()}


def test_describe(client):
    from paper_1011_3583_gb300 import librearr
    d = librearr.describe_permute(4, [512, 512, 512], [2, 1, 0])
    got = client["describe"]
    assert got[0] == "REARR_OK"
    assert librearr.KIND_NAMES[int(got[2])] == d["kind"] == "tile"
    assert (int(got[4]), int(got[6]), int(got[8]), int(got[10])) == (d["rank"], d["cell_bytes"], d["word_bytes"],
                                                                      d["n_tiles"])


def test_rejections(client):
    assert client["bad_perm"] == ["REARR_EINVAL"]
    assert client["pipeline"] == ["REARR_EINVAL"]


def test_dist_plan(client):
    got = client["dist"]
    assert got[:6] == ["REARR_OK", "exchange", "1", "slab", "384", "piece"] and got[6] == "192"
    i = got.index("pack")
    j = got.index("unpack")
    assert got[i + 1:j] == ["4/2", "6/3", "2/0", "2/1"]
    assert got[j + 1:] == ["2/1", "2/0", "4/2", "6/3"]


def test_stencil_and_selftest(client):
    assert client["stencil"] == ["REARR_OK", "shape", "1", "radius", "1"]  # a cross of radius 1
    assert client["selftest"] == ["REARR_OK"]


def test_describe_reorder_and_box(client):
    assert client["reorder"] == ["REARR_OK", "form", "1", "chunks", "64", "16384"]  # REARR_REORDER_SMEM_SCATTER
    assert client["nm"] == ["REARR_OK", "kind", "5"]                                 # REARR_KIND_STRIDED


@pytest.mark.gpu
def test_device_permute_from_c(tmp_path):
    """tests/c_abi/device_client.c: cudaMalloc'd buffers, one rearr_permute of
    a 2 x 3 fp32 matrix, checked in C against the hand-written transpose."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    rbuild.build()
    from paper_1011_3583_gb300 import librearr
    libdir = os.path.dirname(librearr.lib_path())
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(rbuild.nvcc())))
    exe = str(tmp_path / "device_client")
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c_abi", "device_client.c"), "-o", exe,
           "-L", libdir, "-lrearr", "-L", os.path.join(cuda, "lib64"), "-lcudart",
           "-Wl,-rpath," + libdir, "-Wl,-rpath," + os.path.join(cuda, "lib64")]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "device_permute OK", out.stdout + out.stderr
