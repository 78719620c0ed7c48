"""The C ABI from a plain C program (no Python in the call path): the
header compiles as C11 and the program links against libwnnc.so (CPU);
on a GPU it orients a sphere's normals and checks them (tests/c)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "sphere_orient.c")
CUDA = "/usr/local/cuda"


def _build(tmp_path):
    import paper_2405_16634_b300 as W
    W.build_if_needed()
    libdir = os.path.dirname(W.LIB_PATH)
    exe = str(tmp_path / "sphere_orient")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), SRC, "-o", exe, "-L", libdir, "-lwnnc",
           "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-lm", f"-Wl,-rpath,{libdir}",
           f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c_program_compiles_and_links(tmp_path):
    exe = _build(tmp_path)
    assert os.path.exists(exe)


@pytest.mark.gpu
def test_c_program_orients_a_sphere(tmp_path):
    exe = _build(tmp_path)
    r = subprocess.run([exe, "20000"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "outward 20000" in r.stdout
