"""The library is usable from plain C through include/sfb.h alone: a C
program (tests/c_abi_program.c) built with gcc against the header and linked
to lib/libsfb.so runs the host set-up calls of the tiny workload, and what it
prints matches the Python binding on the same workload. No GPU call is made."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import sfb_workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_uses_the_abi():
    import paper_1802_06263_gb300 as sfb
    if not os.path.exists(sfb.library_path()):
        sfb.build()
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = sfb.library_path()
    exe = os.path.join(ROOT, "paper_1802_06263_gb300", "_build", "c_abi_program")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_program.c"), "-o", exe, lib,
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    out = {ln.split()[0]: ln.split()[1:] for ln in r.stdout.splitlines()}
    s = sfb.Solver(W.tiny())
    assert int(out["n_lambda"][0]) == s.n_lambda and int(out["n_darcy"][0]) == s.n_darcy
    assert np.array_equal(np.array(out["eig"], dtype=float), s.eigvals)
    assert int(out["n_pts"][0]) == s.n_pts == 16
    assert abs(float(out["weight_sum"][0]) - 1.0) < 1e-15
    assert int(out["workspace_fp64"][0]) == s.workspace_bytes(sfb.FP64, s.n_pts)
    assert int(out["workspace_mixed"][0]) == s.workspace_bytes(sfb.MIXED, s.n_pts)
    assert tuple(int(v) for v in out["shape"]) == sfb.basis_launch_shape(sfb.MIXED, 0, 0)
    # the binding's ctypes mirrors have the C layouts
    import ctypes
    for key, cls, last in (("layout_problem", sfb.Problem, "source"), ("layout_kl_region", sfb.KLRegion, "n_modes_y"),
                           ("layout_collocation", sfb.Collocation, "m_dim"),
                           ("layout_basis_stats", sfb.BasisStats, "mean_refine_steps")):
        size, off = (int(v) for v in out[key])
        assert ctypes.sizeof(cls) == size, key
        assert getattr(cls, last).offset == off, key
