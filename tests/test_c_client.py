"""The boundary from plain C: tests/c/mf_solve_file.c includes include/mf.h,
links libmf.so and drives create / set_caps / solve / flow / cuts with no
Python in between.  Without a GPU the program must compile and link cleanly
as C99 (the header is self-contained C); on a GPU its flow value and both
cuts must equal the oracle's on seeded instances (inputs from gen/)."""
import os
import subprocess

import numpy as np
import pytest

import __graft_entry__
import oracle
from gen import grids
from paper_1109_1146_gb300 import mf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "mf_solve_file.c")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    __graft_entry__.build()
    libdir = os.path.dirname(mf.LIBPATH)
    exe = str(tmp_path_factory.mktemp("c") / "mf_solve_file")
    subprocess.run(["gcc", "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), SRC,
                    "-L", libdir, "-lmf", f"-Wl,-rpath,{libdir}", "-o", exe], check=True, capture_output=True)
    return exe


def test_client_compiles_and_links_as_c99(client):
    assert os.access(client, os.X_OK)


def test_header_compiles_as_cpp():
    # the extern "C" guards let C++ callers include the header unchanged
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Wextra", "-Werror", "-x", "c++", "-fsyntax-only",
                    os.path.join(ROOT, "include", "mf.h")], check=True, capture_output=True)


def _write(path, inst, tile):
    ndim = 3 if inst.conn == 6 else 2
    hdr = np.array([ndim, inst.conn, *inst.dims, *tile], dtype="<i4")
    with open(path, "wb") as f:
        for a in (hdr, inst.cs, inst.ct, np.asarray(inst.nlink).ravel()):
            f.write(np.ascontiguousarray(a, dtype="<i4").tobytes())


@pytest.mark.gpu
@pytest.mark.parametrize("make,tile", [
    (lambda: grids.segmentation_2d(150, 97, 1, conn=4, hard_seed_frac=0.03), (32, 32, 1)),
    (lambda: grids.segmentation_2d(131, 170, 2, conn=8, hard_seed_frac=0.05), (64, 64, 1)),
    (lambda: grids.volume_3d(45, 30, 21, 3), (32, 8, 4)),
])
def test_client_solves_like_the_oracle(client, tmp_path, make, tile):
    inst = make()
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    _write(fin, inst, tile)
    r = subprocess.run([client, str(fin), str(fout)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    raw = fout.read_bytes()
    flow = int(np.frombuffer(raw[:8], dtype="<i8")[0])
    sweeps = int(np.frombuffer(raw[8:12], dtype="<i4")[0])
    smin = np.frombuffer(raw[12:12 + inst.n], dtype=np.uint8)
    smax = np.frombuffer(raw[12 + inst.n:12 + 2 * inst.n], dtype=np.uint8)
    ref = oracle.solve_instance(inst)
    assert flow == ref["flow"] and sweeps >= 1
    np.testing.assert_array_equal(smin, ref["smin"])
    np.testing.assert_array_equal(smax, ref["smax"])
