"""Shared helpers of the GPU tests: an engine session on cuda:0, model and
contract construction from the synthetic workloads, and the per-path
comparison rule against the oracle."""
from __future__ import annotations

import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2108_03076_gb300 as pc
from conftest import ROOT
from oracle import il_text, mc
from oracle.paths import Market

TIE = 1e-5           # comparisons closer than this (relative) to a tie may flip
RTOL = 1e-5          # per-path tolerance relative to max(|x|, notional)


class Engine:
    """Context on cuda:0 (torch's current stream) plus object bookkeeping."""

    def __init__(self):
        from paper_2108_03076_gb300 import build
        build.build()
        self.stream = torch.cuda.Stream()
        torch.cuda.set_stream(self.stream)
        self.ctx = pc.pc_create(0, self.stream.cuda_stream)
        self.models, self.contracts = [], []

    def model(self, spec) -> int:
        h = pc.pc_model_create(self.ctx, spec.S0, spec.sigma, spec.corr, spec.r, spec.days,
                               getattr(spec, "now", 0), getattr(spec, "history", None) or None,
                               getattr(spec, "hist_days", None) or None)
        self.models.append(h)
        return h

    def contract(self, text: str, tparams=(), p1=0, p2=1) -> int:
        w, k = pc.pc_assemble(text)
        h = pc.pc_load_payoff(self.ctx, w, k, tparams, p1, p2)
        self.contracts.append(h)
        return h

    def paths(self, model, contract, n, seed, offset=0, stream=0):
        """Per-path payoffs (float64 copy of the FP32 values) and the
        kernel's (sum, sumsq, n)."""
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        x = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
        pc.pc_price_paths(model, contract, n, offset, seed, stream, out.data_ptr(), x.data_ptr())
        torch.cuda.synchronize()
        return x[:n].double().cpu().numpy(), out.cpu().numpy()

    def sums(self, model, contract, n, seed, offset=0, stream=0):
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        pc.pc_price_async(model, contract, n, offset, seed, stream, out.data_ptr())
        torch.cuda.synchronize()
        return out.cpu().numpy()

    def close(self):
        for k in self.contracts:
            pc.pc_contract_destroy(k)
        for m in self.models:
            pc.pc_model_destroy(m)
        pc.pc_destroy(self.ctx)


def market(spec) -> Market:
    return Market(**vars(spec))


def tparam_env(tparams):
    return {f"${i}": v for i, v in enumerate(tparams)}


def oracle_paths(text, spec, tparams, n, seed, offset=0, stream=0, paths=None, p1=0, p2=1):
    prog = il_text.parse(text)
    return mc.payoffs(prog, market(spec), tparam_env(tparams), p1, p2, n, seed, stream, offset,
                      paths=paths, with_margins=True)


def compare(x_gpu, x_ref, margins, notional, what=""):
    """Per-path parity: |x_gpu - x_ref| <= RTOL * max(|x_ref|, notional) on
    every path whose comparisons were not within TIE of a tie; on the
    others a differing decision is allowed on at most max(2, 1e-4 N) paths."""
    x_gpu, x_ref = np.asarray(x_gpu), np.asarray(x_ref)
    assert x_gpu.shape == x_ref.shape
    assert np.all(np.isfinite(x_gpu)), what
    tol = RTOL * np.maximum(np.abs(x_ref), notional)
    bad = np.abs(x_gpu - x_ref) > tol
    amb = margins < TIE
    hard = np.nonzero(bad & ~amb)[0]
    assert len(hard) == 0, (what, hard[:5], x_gpu[hard[:5]], x_ref[hard[:5]])
    flips = int((bad & amb).sum())
    assert flips <= max(2, 1e-4 * len(x_ref)), (what, flips)
    return flips


def curand_reference_lib():
    """Build (once) and load the cuRAND Philox helper of tests/cuda."""
    import ctypes
    from paper_2108_03076_gb300.build import cuda_home, ARCH
    src = os.path.join(ROOT, "tests", "cuda", "curand_philox_ref.cu")
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libcurand_philox_ref.so")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        cuda = cuda_home()
        subprocess.run([os.path.join(cuda, "bin", "nvcc"), *ARCH, "-O2", "-Xcompiler", "-fPIC",
                        "-shared", "-cudart", "shared", src, "-o", so], check=True)
    L = ctypes.CDLL(so)
    L.curand_philox_ref.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_void_p, ctypes.c_size_t]
    L.curand_philox_ref.restype = ctypes.c_int
    return L
