"""Accuracy of a DFT stage done as a tensor-core GEMM, against the FP32 codelets.

The optional tensor-core stage would form the length-R sub-DFTs of the row
transforms as a real GEMM [2R x 2R] x [2R x batch], with the operands split
into BF16 parts (three terms, all nine cross products) or TF32 parts (big +
small, three cross products: the "3xTF32" correction), accumulating in FP32.
It is to be kept only if its error beats the FP32 path.  This test measures
both on the same inputs in an idealised emulation: every partial product is
exact and the accumulation is FP32 in a fixed order, so real tensor cores can
only do as well or worse.  The FP32 path is the generated codelet itself,
evaluated statement by statement in FP32.  Reference: the FP64 DFT."""
import importlib.util
import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2012_04838_gb300", "csrc")


def _generator():
    spec = importlib.util.spec_from_file_location("gen_codelets", os.path.join(CSRC, "gen_codelets.py"))
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    return g


G = _generator()
f32 = np.float32


class _C:
    def __init__(self, v):
        self.x, self.y = f32(v.real), f32(v.imag)


def codelet_fp32(src, x):
    """One generated codelet body executed in FP32 (each operation rounded)."""
    env = {"x": [_C(v) for v in x]}
    body = src[src.index("{  //"):]
    for line in body.splitlines()[1:]:
        line = line.strip()
        if not line or line.startswith("}"):
            continue
        if line.startswith("const T "):
            for decl in line[len("const T "):].rstrip(";").split(", "):
                name, expr = decl.split(" = ", 1)
                env[name] = f32(eval(expr.replace("T(", "f32("), {"f32": f32}, env))
        else:
            for stmt in line.rstrip(";").split("; "):
                m = re.match(r"x\[(\d+)\]\.([xy]) = (.*)", stmt)
                k, c, expr = int(m.group(1)), m.group(2), m.group(3)
                setattr(env["x"][k], c, f32(eval(expr.replace("T(", "f32("), {"f32": f32}, env)))
    return np.array([complex(v.x, v.y) for v in env["x"]])


def to_bf16(a):
    """Round FP32 values to BF16 (nearest, ties to even), returned as FP32."""
    b = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def to_tf32(a):
    """Round FP32 values to TF32 (10 fraction bits, nearest, ties to even)."""
    b = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0xFFF + ((b >> 13) & 1)) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32)


def split(a, rnd, terms):
    parts, r = [], np.asarray(a, dtype=np.float32)
    for _ in range(terms):
        p = rnd(r)
        parts.append(p)
        r = (r - p).astype(np.float32)
    return parts


def gemm_fp32(A, B):
    """A @ B with exact products accumulated in FP32, in index order."""
    out = np.zeros((A.shape[0], B.shape[1]), dtype=np.float32)
    for k in range(A.shape[1]):
        out = (out + (A[:, k:k + 1].astype(np.float64) * B[k:k + 1, :]).astype(np.float32)).astype(np.float32)
    return out


def dft_gemm(x, R, s, rnd, terms, pairs):
    """The length-R DFT of the columns of x as the real GEMM [[C, -S], [S, C]]
    times [re; im], operands split by `rnd` into `terms` parts and the cross
    products (i, j) in `pairs` summed in FP32."""
    n = np.arange(R)
    ang = s * 2.0 * np.pi * np.outer(n, n) / R
    W = np.block([[np.cos(ang), -np.sin(ang)], [np.sin(ang), np.cos(ang)]]).astype(np.float32)
    X = np.vstack([x.real, x.imag]).astype(np.float32)
    Wp, Xp = split(W, rnd, terms), split(X, rnd, terms)
    acc = np.zeros((2 * R, x.shape[1]), dtype=np.float32)
    for i, j in pairs:
        acc = (acc + gemm_fp32(Wp[i], Xp[j])).astype(np.float32)
    return acc[:R].astype(np.float64) + 1j * acc[R:].astype(np.float64)


def rel_err(got, ref):
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("R", [16, 32])
def test_tensor_core_dft_stage_is_fp32_level_like_the_codelet(R):
    rng = np.random.default_rng(R)
    batch = 64
    x = (rng.standard_normal((R, batch)) + 1j * rng.standard_normal((R, batch))).astype(np.complex64)
    x = x.astype(np.complex128)
    s = -1
    n = np.arange(R)
    ref = np.exp(s * 2j * np.pi * np.outer(n, n) / R) @ x
    src = G.codelet(R, s)
    e_codelet = rel_err(np.stack([codelet_fp32(src, x[:, b]) for b in range(batch)], axis=1), ref)
    bf16_all = [(i, j) for i in range(3) for j in range(3)]
    e_bf16 = rel_err(dft_gemm(x, R, s, to_bf16, 3, bf16_all), ref)
    e_tf32 = rel_err(dft_gemm(x, R, s, to_tf32, 2, [(0, 0), (0, 1), (1, 0)]), ref)
    print(f"R={R}: FP32 codelet {e_codelet:.3e}, split-BF16 x9 {e_bf16:.3e}, 3xTF32 {e_tf32:.3e}")
    # all three are FP32-level transforms ...
    for e in (e_codelet, e_bf16, e_tf32):
        assert 1e-8 < e < 1e-6
    # ... and even the idealised GEMM forms are at most marginally more
    # accurate (measured: split-BF16 about 15% below the codelet, 3xTF32 above
    # it), far from an accuracy gain that would pay for nine (or three) GEMM
    # passes per DFT stage
    assert min(e_bf16, e_tf32) > 0.5 * e_codelet
