"""The C ABI from plain C: a C99 program (tests/c_client/host_calls.c)
compiles against include/hmc.h, links libhmc.so and calls the entry points
that need no GPU.  Its sizes match the layouts, its filter and rooted
coefficients match the oracle's exact rational series, and a NULL context is
refused."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import coeffs as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def output(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_1805_03560_gb300 import build
    build.build()
    lib_dir = os.path.join(ROOT, "paper_1805_03560_gb300")
    exe = str(tmp_path_factory.mktemp("c_client") / "host_calls")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_client", "host_calls.c"),
                    "-L", lib_dir, "-lhmc", "-Wl,-rpath," + lib_dir, "-o", exe], check=True)
    run = subprocess.run([exe], check=True, capture_output=True, text=True)
    rows = {}
    for line in run.stdout.splitlines():
        key, *rest = line.split(" ", 1)
        rows.setdefault(key, []).append(rest[0] if rest else "")
    return rows


def test_sizes_from_c(output):
    Vh = 48 * 24 ** 3 // 2
    assert int(output["spinor_bytes_f32"][0]) == Vh * 96
    assert int(output["gauge_bytes_f32_12"][0]) == 2 * Vh * 4 * 48
    assert int(output["algebra_bytes"][0]) == 2 * Vh * 4 * 8 * 8
    assert int(output["spinor_bytes_odd"][0]) == 0


def _indexed(rows):
    return np.array([float(v.split()[1]) for v in rows])


def test_filter_coefficients_from_c(output):
    assert output["filter_status"] == ["0"] and output["filter_bad"] == ["1"]
    b, alpha, _ = C.filter_coeffs(2, 29)
    assert abs(float(output["filter_alpha"][0]) - alpha) < 1e-15
    assert np.allclose(_indexed(output["filter_b"]), b, rtol=1e-14, atol=1e-300)
    assert np.allclose(_indexed(output["filter_c"]), C.heatbath_coeffs(2, 29), rtol=1e-14,
                       atol=1e-300)


def test_rooted_coefficients_from_c(output):
    assert output["rooted_status"] == ["0"]
    alpha, _, polys = C.rooted_coeffs(2, 2, (6, 12), 20)
    assert abs(float(output["rooted_alpha"][0]) - alpha) <= 1e-13 * abs(alpha)
    want = [float(x) for p in polys for x in p]
    assert np.allclose(_indexed(output["rooted_poly"]), want, rtol=1e-13, atol=1e-16)


def test_null_context_from_c(output):
    assert output["null_ctx"] == ["1"]  # HMC_EINVAL
    assert output["null_ctx_error"] == ["context is NULL"]
