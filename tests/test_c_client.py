"""The C ABI from plain C: tests/c_client.c, compiled with gcc against
include/permanova.h and linked to libpermanova.so, builds and links on any
machine (no GPU needed) and, on the GPU, gets s_W through the host-buffer
entry point and checks it against the statistic's definition, then checks
the error path (EINVAL with a message, the context still usable)."""
import os
import shutil
import subprocess

import pytest

import paper_2505_04556_gb300 as pm

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

pytestmark = pytest.mark.skipif(
    shutil.which("gcc") is None or (shutil.which("nvcc") is None and not os.path.exists(pm.LIB_PATH)),
    reason="gcc and the library (or nvcc to build it) are needed")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    pm.build()
    exe = str(tmp_path_factory.mktemp("c_client") / "c_client")
    libdir = os.path.dirname(pm.LIB_PATH)
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "c_client.c"), "-o", exe, "-L", libdir, "-lpermanova",
           f"-Wl,-rpath,{libdir}", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_c_client_builds_and_links(client):
    assert os.access(client, os.X_OK)


@pytest.mark.gpu
def test_c_client_runs_on_the_gpu(client):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([client], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c client OK" in r.stdout
