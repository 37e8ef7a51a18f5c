"""The in-register DFT codelets of the GPU path, checked on the CPU.

codelets.cuh must be exactly what gen_codelets.py emits, and every emitted
codelet (full, and with a range of inputs known to be zero) is evaluated here
statement by statement in Python and compared with numpy's FFT, the
unnormalised sum X[k] = sum_n x[n] exp(s 2 pi i n k / R)."""
import importlib.util
import io
import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2012_04838_gb300", "csrc")


def load_generator():
    spec = importlib.util.spec_from_file_location("gen_codelets", os.path.join(CSRC, "gen_codelets.py"))
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    return g


G = load_generator()


def test_committed_codelets_match_generator():
    out = io.StringIO()
    G.main(out)
    with open(os.path.join(CSRC, "codelets.cuh")) as f:
        assert f.read() == out.getvalue()


class _C:
    def __init__(self, v):
        self.x, self.y = v.real, v.imag


def run_codelet(src: str, x: np.ndarray) -> np.ndarray:
    """Execute one generated codelet body on x (complex), in float64."""
    env = {"T": float, "x": [_C(v) for v in x]}
    body = src[src.index("{  //"):]
    for line in body.splitlines()[1:]:
        line = line.strip()
        if not line or line.startswith("}"):
            continue
        if line.startswith("const T "):
            for decl in line[len("const T "):].rstrip(";").split(", "):
                name, expr = decl.split(" = ", 1)
                env[name] = eval(expr.replace("T(", "float("), {"float": float}, env)
        else:
            for stmt in line.rstrip(";").split("; "):
                m = re.match(r"x\[(\d+)\]\.([xy]) = (.*)", stmt)
                k, c, expr = int(m.group(1)), m.group(2), m.group(3)
                setattr(env["x"][k], c, eval(expr.replace("T(", "float("), {"float": float}, env))
    return np.array([complex(v.x, v.y) for v in env["x"]])


def reference_dft(x, s):
    R = len(x)
    n = np.arange(R)
    return np.exp(s * 2j * np.pi * np.outer(n, n) / R) @ x


@pytest.mark.parametrize("R", G.SIZES)
@pytest.mark.parametrize("s", [-1, 1])
def test_codelet_is_the_dft(R, s):
    rng = np.random.default_rng(R * 10 + (s > 0))
    x = rng.standard_normal(R) + 1j * rng.standard_normal(R)
    got = run_codelet(G.codelet(R, s), x)
    np.testing.assert_allclose(got, reference_dft(x, s), rtol=0, atol=1e-12 * R)


@pytest.mark.parametrize("N", sorted(G.PLANS))
def test_zero_input_codelets(N):
    z = G.zero_range(N)
    if z is None:
        pytest.skip("no input of the first DFT is zero for every column")
    R, z0, z1 = z
    R1, R2 = G.PLANS[N]
    K = (N - 1) // 3
    # every skipped input really is in the zero band for every column n2
    for n1 in range(z0, z1 + 1):
        for n2 in range(R2):
            p = R2 * n1 + n2
            assert K < p < N - K
    rng = np.random.default_rng(N)
    x = rng.standard_normal(R) + 1j * rng.standard_normal(R)
    x[z0:z1 + 1] = 0
    got = run_codelet(G.codelet(R, 1, (z0, z1)), x)
    np.testing.assert_allclose(got, reference_dft(x, 1), rtol=0, atol=1e-12 * R)
    # the pruned codelet never reads the zero inputs: garbage there changes nothing
    y = x.copy()
    y[z0:z1 + 1] = 1e30
    np.testing.assert_array_equal(run_codelet(G.codelet(R, 1, (z0, z1)), y), got)
