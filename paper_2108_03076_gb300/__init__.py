"""Python binding of the payoff-expression Monte Carlo engine (``libpc.so``).

Argument marshalling only: every function forwards to the C entry point of
the same name declared in ``include/pc.h``; all computation runs in the
library's CUDA kernels.  Device buffers are passed as integer addresses
(e.g. ``torch.Tensor.data_ptr()``), CUDA streams as ``cudaStream_t`` values
(e.g. ``torch.cuda.current_stream().cuda_stream``).  A non-OK status raises
``PcError`` carrying the status code and ``pc_last_error()``.

The library must have been built (``paper_2108_03076_gb300.build.build()``);
there is no fallback implementation.

Submodules: ``build`` (nvcc build of libpc.so), ``merge`` (host merge of
per-process sums), ``autograd`` (pathwise-sensitivity autograd function),
``learned_cv`` (training set, network and tables of the learned control
variate).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpc.so")

PC_OK = 0
STATUS = {0: "PC_OK", -1: "PC_EINVAL", -2: "PC_EBYTECODE", -3: "PC_ETPARAM", -4: "PC_ERANGE",
          -5: "PC_ENOTPD", -6: "PC_ENOMEM", -7: "PC_ECUDA", -8: "PC_ETIMEOUT",
          -9: "PC_EDEVICE", -10: "PC_ELIMIT", -11: "PC_ESYNTAX"}
globals().update({v: k for k, v in STATUS.items()})

MAX_UNDERLYINGS = 4


class PcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class ModelDesc(C.Structure):
    _fields_ = [("d", C.c_int32), ("S0", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
                ("corr", C.POINTER(C.c_double)), ("r", C.c_double), ("n_dates", C.c_int32),
                ("day", C.POINTER(C.c_int32)), ("t_now", C.c_int32), ("n_hist", C.c_int32),
                ("history", C.POINTER(C.c_double)), ("hist_day", C.POINTER(C.c_int32))]


class ModelInfo(C.Structure):
    _fields_ = [("d", C.c_int32), ("n_dates", C.c_int32), ("n_hist", C.c_int32),
                ("t_now", C.c_int32), ("bridge_levels", C.c_int32), ("bridge_stack", C.c_int32),
                ("philox_blocks", C.c_int32), ("box_muller_pairs", C.c_int32)]


class BatchConfig(C.Structure):
    _fields_ = [("block", C.c_int32), ("unit_split", C.c_int32)]


class BatchInfo(C.Structure):
    _fields_ = [("n_contracts", C.c_uint64), ("n_tiles", C.c_uint64), ("n_units", C.c_uint64),
                ("n_groups", C.c_int32), ("tuned", C.c_int32), ("config", BatchConfig),
                ("paths_per_thread", C.c_double), ("last_ms", C.c_double), ("n_specialised", C.c_int32)]


class MlpInfo(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("widths", C.c_int32 * 9), ("n_params", C.c_uint64),
                ("max_batch", C.c_uint64), ("steps", C.c_uint64)]


CV_MAX_DATES = 32


class CvDesc(C.Structure):
    _fields_ = [("d", C.c_int32), ("n", C.c_int32), ("grid", C.c_int32), ("ref", C.c_float * 3),
                ("call_level", C.c_float), ("ki_level", C.c_float), ("coupon", C.c_float),
                ("lo", (C.c_float * 3) * CV_MAX_DATES), ("h", (C.c_float * 3) * CV_MAX_DATES),
                ("delta0", C.c_float * 3), ("beta", C.c_float), ("beta2", C.c_float),
                ("use_gamma", C.c_int32), ("delta0_on_device", C.c_int32)]


class LaunchInfo(C.Structure):
    _fields_ = [("window", C.c_int32), ("hbm_window", C.c_int32), ("block", C.c_int32),
                ("grid", C.c_int32), ("smem_bytes", C.c_uint64), ("hbm_window_bytes", C.c_uint64),
                ("window_bytes_written_per_path_date", C.c_uint64)]


WINDOW_AUTO, WINDOW_SHARED, WINDOW_HBM = 0, 1, 2
MLP_GEMM_AUTO, MLP_GEMM_MMA_SYNC = 0, 1
JIT_MAX_INSNS = 384  # longer programs are interpreted with pc_set_jit on (pc.h)


class ProgramInfo(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_insn", C.c_int32), ("max_stack", C.c_int32),
                ("result_is_real", C.c_int32), ("n_loops", C.c_int32),
                ("n_tparams_used", C.c_int32)]


_lib: Optional[C.CDLL] = None
VP, U64, U32, I32, SZ, DBL = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int32, C.c_size_t, C.c_double
PD, PU32, PI32, PF = C.POINTER(C.c_double), C.POINTER(C.c_uint32), C.POINTER(C.c_int32), C.POINTER(C.c_float)

_SIGS = {
    "pc_create": [C.POINTER(VP), C.c_int, VP],
    "pc_destroy": [VP],
    "pc_last_error": [VP],
    "pc_model_create": [VP, C.POINTER(ModelDesc), C.POINTER(VP)],
    "pc_model_destroy": [VP],
    "pc_model_query": [VP, C.POINTER(ModelInfo)],
    "pc_load_payoff": [VP, PU32, SZ, PD, SZ, PI32, SZ, I32, I32, C.POINTER(VP)],
    "pc_load_payoffs": [VP, SZ, PU32, C.POINTER(SZ), PD, C.POINTER(SZ), PI32, C.POINTER(SZ), I32, I32,
                        C.POINTER(VP)],
    "pc_contract_destroy": [VP],
    "pc_verify_payoff": [PU32, SZ, PD, SZ, PI32, SZ, C.POINTER(ProgramInfo)],
    "pc_assemble": [C.c_char_p, PU32, SZ, C.POINTER(SZ), PD, SZ, C.POINTER(SZ), C.c_char_p, SZ],
    "pc_price": [VP, VP, U64, U64, PD, PD],
    "pc_price_async": [VP, VP, U64, U64, U64, U32, VP],
    "pc_price_paths": [VP, VP, U64, U64, U64, U32, VP, VP],
    "pc_price_noalloc": [VP, VP, U64, U64, U64, U32, VP],
    "pc_cut_payoff": [PU32, SZ, PD, SZ, PU32, SZ, C.POINTER(SZ), PD, SZ, C.POINTER(SZ)],
    "pc_set_timeout": [VP, DBL],
    "pc_cv_labels": [SZ, I32, PD, PD, DBL, I32, PF],
    "pc_debug_fail_allocations": [VP, I32],
    "pc_debug_set_status": [VP, I32],
    "pc_debug_mlp_withhold_tma": [VP, I32],
    "pc_greeks_adjoint": [VP, VP, U64, U64, PD, PD, PD, PD],
    "pc_greeks_adjoint_async": [VP, VP, U64, U64, U64, U32, VP],
    "pc_debug_adjoint_paths": [VP, VP, U64, U64, U64, VP, VP],
    "pc_price_batch": [SZ, C.POINTER(VP), C.POINTER(VP), C.POINTER(U64), U64, PD, PD],
    "pc_set_window_mode": [VP, C.c_int32],
    "pc_set_jit": [VP, C.c_int32],
    "pc_debug_set_jit_pairs": [VP, C.c_int32],
    "pc_debug_set_cv_min_blocks": [VP, C.c_int32],
    "pc_jit_compile": [VP, VP],
    "pc_debug_jit_compile": [PU32, SZ, PD, SZ, PI32, SZ, I32, I32, I32, I32, C.POINTER(SZ)],
    "pc_debug_jit_source": [PU32, SZ, PD, SZ, PI32, SZ, I32, I32, I32, I32, C.c_char_p, SZ, C.POINTER(SZ)],
    "pc_price_info": [VP, VP, U64, C.POINTER(LaunchInfo)],
    "pc_batch_create": [SZ, C.POINTER(VP), C.POINTER(VP), C.POINTER(U64), U64,
                        C.POINTER(BatchConfig), C.POINTER(VP)],
    "pc_batch_tune": [VP, C.c_int32],
    "pc_batch_launch": [VP],
    "pc_batch_results": [VP, PD, PD, PD],
    "pc_batch_query": [VP, C.POINTER(BatchInfo)],
    "pc_batch_set_single_launch": [VP, C.c_int32],
    "pc_batch_destroy": [VP],
    "pc_mlp_create": [VP, C.POINTER(C.c_int32), C.c_int32, U64, U64, C.POINTER(VP)],
    "pc_mlp_destroy": [VP],
    "pc_mlp_query": [VP, C.POINTER(MlpInfo)],
    "pc_mlp_set_params": [VP, C.POINTER(C.c_float), SZ],
    "pc_mlp_get_params": [VP, C.POINTER(C.c_float), SZ],
    "pc_mlp_forward": [VP, VP, SZ, VP],
    "pc_mlp_set_gemm": [VP, C.c_int32],
    "pc_mlp_gemm_info": [VP, C.POINTER(C.c_int32)],
    "pc_mlp_gradients": [VP, VP, VP, C.POINTER(C.c_float), SZ, VP, PD],
    "pc_mlp_train": [VP, VP, VP, SZ, C.POINTER(C.c_float), SZ, C.c_int32, C.c_float, U64, PD],
    "pc_cv_grid": [VP, C.c_int32, C.c_float, C.POINTER(CvDesc)],
    "pc_cv_table_size": [C.POINTER(CvDesc), C.POINTER(SZ)],
    "pc_cv_tables": [VP, VP, C.POINTER(CvDesc), VP, SZ],
    "pc_cv_tables_async": [VP, VP, C.POINTER(CvDesc), VP, SZ],
    "pc_price_cv": [VP, VP, C.POINTER(CvDesc), VP, U64, U64, PD],
    "pc_cv_beta": [VP, VP, C.POINTER(CvDesc), VP, U64, U64, PD],
    "pc_debug_cv_paths": [VP, VP, C.POINTER(CvDesc), VP, U64, U64, VP],
    "pc_greeks": [VP, VP, U64, U64, PD, PD, PD, PD],
    "pc_debug_philox": [VP, VP, U32, U32, VP, SZ],
    "pc_debug_paths": [VP, U64, U64, U64, U32, VP],
    "pc_debug_greeks_paths": [VP, VP, U64, U64, U64, I32, VP, VP],
    "pc_debug_program": [PU32, SZ, PD, SZ, PI32, SZ, I32, I32, PU32, SZ, C.POINTER(SZ),
                         C.POINTER(SZ)],
    "pc_debug_bridge": [C.POINTER(ModelDesc), PI32, PU32, SZ, C.POINTER(SZ)],
}
EXPORTED = tuple(_SIGS)


def lib() -> C.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2108_03076_gb300.build.build() (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_char_p if name == "pc_last_error" else C.c_int32
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != PC_OK:
        raise PcError(status, lib().pc_last_error(None).decode(errors="replace"))


def _arr(a, dtype):
    a = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    return a


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a.size else None


# ---------------------------------------------------------------------------
# Context / model / contract
# ---------------------------------------------------------------------------


def pc_create(device: int = 0, stream: int | None = None) -> int:
    h = VP()
    _check(lib().pc_create(C.byref(h), device, VP(stream) if stream else None))
    return h.value


def pc_destroy(ctx: int) -> None:
    _check(lib().pc_destroy(VP(ctx)))


def pc_last_error() -> str:
    return lib().pc_last_error(None).decode(errors="replace")


def _model_desc(S0, sigma, corr, r, days, t_now=0, history=None, hist_days=None):
    """A ModelDesc plus the arrays it points into (kept alive together)."""
    keep = [_arr(S0, np.float64), _arr(sigma, np.float64), _arr(corr, np.float64).reshape(-1),
            _arr(days, np.int32),
            _arr(history if history is not None else [], np.float64).reshape(-1),
            _arr(hist_days if hist_days is not None else [], np.int32)]
    S0a, sga, ca, da, ha, hda = keep
    desc = ModelDesc(len(S0a), _ptr(S0a, C.c_double), _ptr(sga, C.c_double), _ptr(ca, C.c_double),
                     float(r), len(da), _ptr(da, C.c_int32), int(t_now), len(hda),
                     _ptr(ha, C.c_double), _ptr(hda, C.c_int32))
    return desc, keep


def pc_model_create(ctx: int, S0: Sequence[float], sigma: Sequence[float],
                    corr: Sequence[Sequence[float]], r: float, days: Sequence[int],
                    t_now: int = 0, history: Sequence[Sequence[float]] | None = None,
                    hist_days: Sequence[int] | None = None) -> int:
    desc, _keep = _model_desc(S0, sigma, corr, r, days, t_now, history, hist_days)
    h = VP()
    _check(lib().pc_model_create(VP(ctx), C.byref(desc), C.byref(h)))
    return h.value


def pc_model_query(model: int) -> ModelInfo:
    info = ModelInfo()
    _check(lib().pc_model_query(VP(model), C.byref(info)))
    return info


def pc_model_destroy(model: int) -> None:
    _check(lib().pc_model_destroy(VP(model)))


def pc_assemble(text: str) -> Tuple[np.ndarray, np.ndarray]:
    """Textual IL -> (bytecode words uint32, real literals float64)."""
    nw, nk = SZ(0), SZ(0)
    err = C.create_string_buffer(512)
    st = lib().pc_assemble(text.encode(), None, 0, C.byref(nw), None, 0, C.byref(nk), err, 512)
    if st not in (PC_OK, -10):
        raise PcError(st, err.value.decode(errors="replace"))
    w = np.zeros(nw.value, np.uint32)
    k = np.zeros(nk.value, np.float64)
    _check(lib().pc_assemble(text.encode(), _ptr(w, C.c_uint32), w.size, C.byref(nw),
                             _ptr(k, C.c_double), k.size, C.byref(nk), err, 512))
    return w, k


def pc_cut_payoff(words, consts) -> Tuple[np.ndarray, np.ndarray]:
    """cutPayoff (Sec. 4.1) of a bytecode program: (words, consts)."""
    w = _arr(words, np.uint32)
    k = _arr(consts, np.float64)
    nw, nk = C.c_size_t(0), C.c_size_t(0)
    cap_w, cap_k = 2 * w.size + 64, k.size + 1
    ow, ok = np.zeros(cap_w, np.uint32), np.zeros(cap_k, np.float64)
    while True:
        st = lib().pc_cut_payoff(_ptr(w, C.c_uint32), w.size, _ptr(k, C.c_double), k.size,
                                 _ptr(ow, C.c_uint32), cap_w, C.byref(nw), _ptr(ok, C.c_double), cap_k,
                                 C.byref(nk))
        if st == PC_ELIMIT and (nw.value > cap_w or nk.value > cap_k):
            cap_w, cap_k = nw.value, nk.value
            ow, ok = np.zeros(cap_w, np.uint32), np.zeros(cap_k, np.float64)
            continue
        _check(st)
        return ow[:nw.value].copy(), ok[:nk.value].copy()


def pc_verify_payoff(words, consts, tparams=()) -> ProgramInfo:
    w, k, t = _arr(words, np.uint32), _arr(consts, np.float64), _arr(tparams, np.int32)
    info = ProgramInfo()
    _check(lib().pc_verify_payoff(_ptr(w, C.c_uint32), w.size, _ptr(k, C.c_double), k.size,
                                  _ptr(t, C.c_int32), t.size, C.byref(info)))
    return info


def pc_load_payoff(ctx: int, words, consts, tparams=(), p1: int = 0, p2: int = 1) -> int:
    w, k, t = _arr(words, np.uint32), _arr(consts, np.float64), _arr(tparams, np.int32)
    h = VP()
    _check(lib().pc_load_payoff(VP(ctx), _ptr(w, C.c_uint32), w.size, _ptr(k, C.c_double), k.size,
                                _ptr(t, C.c_int32), t.size, int(p1), int(p2), C.byref(h)))
    return h.value


class ProgramSet:
    """Programs concatenated once for pc_load_payoffs: a list of
    (words, consts, tparams)."""

    def __init__(self, programs):
        progs = list(programs)
        self.n = len(progs)
        parts = [(_arr(w, np.uint32), _arr(k, np.float64), _arr(t, np.int32)) for w, k, t in progs]
        off = lambda xs: np.concatenate([[0], np.cumsum([x.size for x in xs])]).astype(np.uintp)  # noqa: E731
        self.words = np.ascontiguousarray(np.concatenate([p[0] for p in parts]) if parts else np.zeros(0, np.uint32))
        self.consts = np.ascontiguousarray(np.concatenate([p[1] for p in parts]) if parts else np.zeros(0))
        self.params = np.ascontiguousarray(np.concatenate([p[2] for p in parts]) if parts else np.zeros(0, np.int32))
        self.word_off = off([p[0] for p in parts])
        self.const_off = off([p[1] for p in parts])
        self.param_off = off([p[2] for p in parts])


def pc_load_payoffs(ctx: int, programs, p1: int = 0, p2: int = 1):
    """Load many programs in one call (a ProgramSet, or a list of
    (words, consts, tparams)); returns the contract handles."""
    ps = programs if isinstance(programs, ProgramSet) else ProgramSet(programs)
    out = (VP * max(ps.n, 1))()
    szp = lambda a: a.ctypes.data_as(C.POINTER(SZ))  # noqa: E731
    _check(lib().pc_load_payoffs(VP(ctx), ps.n, _ptr(ps.words, C.c_uint32), szp(ps.word_off),
                                 _ptr(ps.consts, C.c_double), szp(ps.const_off), _ptr(ps.params, C.c_int32),
                                 szp(ps.param_off), int(p1), int(p2), out))
    return [out[i] for i in range(ps.n)]


def pc_contract_destroy(contract: int) -> None:
    _check(lib().pc_contract_destroy(VP(contract)))


# ---------------------------------------------------------------------------
# Pricing
# ---------------------------------------------------------------------------


def pc_price(model: int, contract: int, n_paths: int, seed: int) -> Tuple[float, float]:
    p, s = DBL(), DBL()
    _check(lib().pc_price(VP(model), VP(contract), n_paths, seed, C.byref(p), C.byref(s)))
    return p.value, s.value


def pc_price_async(model: int, contract: int, n_paths: int, path_offset: int, seed: int,
                   stream_id: int, d_out: int) -> None:
    _check(lib().pc_price_async(VP(model), VP(contract), n_paths, path_offset, seed, stream_id,
                                VP(d_out)))


def pc_price_paths(model: int, contract: int, n_paths: int, path_offset: int, seed: int,
                   stream_id: int, d_out: int, d_payoffs: int) -> None:
    _check(lib().pc_price_paths(VP(model), VP(contract), n_paths, path_offset, seed, stream_id,
                                VP(d_out), VP(d_payoffs)))


def pc_price_noalloc(model: int, contract: int, n_paths: int, path_offset: int, seed: int,
                     stream_id: int, d_out: int) -> None:
    """pc_price_async without device allocation: scratch comes from the
    library's fixed device array (at most NOALLOC_MAX_PATHS paths per call;
    calls that overlap on the GPU race)."""
    _check(lib().pc_price_noalloc(VP(model), VP(contract), n_paths, path_offset, seed, stream_id,
                                  VP(d_out)))


NOALLOC_MAX_PATHS = 1 << 24


def pc_set_window_mode(ctx: int, mode: int) -> None:
    _check(lib().pc_set_window_mode(VP(ctx), int(mode)))


def pc_set_timeout(ctx: int, seconds: float) -> None:
    _check(lib().pc_set_timeout(VP(ctx), float(seconds)))


def pc_debug_fail_allocations(ctx: int, count: int) -> None:
    _check(lib().pc_debug_fail_allocations(VP(ctx), int(count)))


def pc_debug_set_status(ctx: int, value: int) -> None:
    _check(lib().pc_debug_set_status(VP(ctx), int(value)))


def pc_debug_mlp_withhold_tma(net: int, on: bool) -> None:
    _check(lib().pc_debug_mlp_withhold_tma(VP(net), int(bool(on))))


def pc_debug_set_jit_pairs(ctx: int, pairs: int) -> None:
    _check(lib().pc_debug_set_jit_pairs(VP(ctx), int(pairs)))


def pc_debug_set_cv_min_blocks(ctx: int, blocks: int) -> None:
    _check(lib().pc_debug_set_cv_min_blocks(VP(ctx), int(blocks)))


def pc_set_jit(ctx: int, enabled: bool) -> None:
    _check(lib().pc_set_jit(VP(ctx), 1 if enabled else 0))


def pc_jit_compile(model: int, contract: int) -> None:
    _check(lib().pc_jit_compile(VP(model), VP(contract)))


def pc_debug_jit_compile(words, consts, tparams=(), d: int = 1, p1: int = 0, p2: int = 1, kind: int = 0) -> int:
    """Host-only: compile a specialised kernel of a program (kind 0 pricing,
    1 per-path pricing, 2 / 3 the same with the window in HBM, 16 + mode
    control variate, 32 / 33 sensitivities); cubin bytes."""
    w, k, t = _arr(words, np.uint32), _arr(consts, np.float64), _arr(tparams, np.int32)
    n = SZ(0)
    _check(lib().pc_debug_jit_compile(_ptr(w, C.c_uint32), w.size, _ptr(k, C.c_double), k.size,
                                      _ptr(t, C.c_int32), t.size, p1, p2, d, int(kind), C.byref(n)))
    return n.value


def pc_debug_jit_source(words, consts, tparams=(), d: int = 1, p1: int = 0, p2: int = 1, kind: int = 0) -> str:
    """Host-only: the CUDA source of a specialised kernel (as handed to
    NVRTC; it includes the library's device headers by name)."""
    w, k, t = _arr(words, np.uint32), _arr(consts, np.float64), _arr(tparams, np.int32)
    n = SZ(0)
    args = (_ptr(w, C.c_uint32), w.size, _ptr(k, C.c_double), k.size, _ptr(t, C.c_int32), t.size,
            p1, p2, d, int(kind))
    _check(lib().pc_debug_jit_source(*args, None, 0, C.byref(n)))
    buf = C.create_string_buffer(n.value + 1)
    _check(lib().pc_debug_jit_source(*args, buf, n.value + 1, C.byref(n)))
    return buf.value.decode()


def pc_price_info(model: int, contract: int, n_paths: int) -> LaunchInfo:
    info = LaunchInfo()
    _check(lib().pc_price_info(VP(model), VP(contract), int(n_paths), C.byref(info)))
    return info


def _batch_arrays(models, contracts, n_paths):
    n = len(contracts)
    if len(models) != n or len(n_paths) != n:
        raise ValueError("models, contracts and n_paths must have the same length")
    M = (VP * n)(*[VP(m) for m in models])
    K = (VP * n)(*[VP(k) for k in contracts])
    N = (U64 * n)(*[int(x) for x in n_paths])
    return n, M, K, N


def pc_price_batch(models: Sequence[int], contracts: Sequence[int], n_paths: Sequence[int],
                   seed: int) -> Tuple[np.ndarray, np.ndarray]:
    n, M, K, N = _batch_arrays(models, contracts, n_paths)
    price, se = np.zeros(n), np.zeros(n)
    _check(lib().pc_price_batch(n, M, K, N, seed, _ptr(price, C.c_double), _ptr(se, C.c_double)))
    return price, se


def pc_batch_create(models: Sequence[int], contracts: Sequence[int], n_paths: Sequence[int],
                    seed: int, block: Optional[int] = None, unit_split: Optional[int] = None) -> int:
    n, M, K, N = _batch_arrays(models, contracts, n_paths)
    cfg = None
    if block is not None or unit_split is not None:
        cfg = C.byref(BatchConfig(block or 128, unit_split or 32))
    h = VP()
    _check(lib().pc_batch_create(n, M, K, N, seed, cfg, C.byref(h)))
    return h.value


def pc_batch_tune(plan: int, reps: int = 2) -> None:
    _check(lib().pc_batch_tune(VP(plan), int(reps)))


def pc_batch_launch(plan: int) -> None:
    _check(lib().pc_batch_launch(VP(plan)))


def pc_batch_results(plan: int, n: int, sums: bool = False):
    """(price[n], stderr[n]) or, with sums, (price, stderr, sums[n, 3])."""
    price, se = np.zeros(n), np.zeros(n)
    out = np.zeros(3 * n) if sums else None
    _check(lib().pc_batch_results(VP(plan), _ptr(price, C.c_double), _ptr(se, C.c_double),
                                  _ptr(out, C.c_double) if sums else None))
    return (price, se, out.reshape(n, 3)) if sums else (price, se)


def pc_batch_set_single_launch(plan: int, enabled: bool) -> None:
    _check(lib().pc_batch_set_single_launch(VP(plan), 1 if enabled else 0))


def pc_batch_query(plan: int) -> BatchInfo:
    info = BatchInfo()
    _check(lib().pc_batch_query(VP(plan), C.byref(info)))
    return info


def pc_batch_destroy(plan: int) -> None:
    _check(lib().pc_batch_destroy(VP(plan)))


def pc_mlp_create(ctx: int, widths: Sequence[int], max_batch: int, seed: int = 1) -> int:
    w = _arr(widths, np.int32)
    h = VP()
    _check(lib().pc_mlp_create(VP(ctx), _ptr(w, C.c_int32), w.size, int(max_batch), int(seed), C.byref(h)))
    return h.value


def pc_mlp_destroy(net: int) -> None:
    _check(lib().pc_mlp_destroy(VP(net)))


def pc_mlp_query(net: int) -> MlpInfo:
    info = MlpInfo()
    _check(lib().pc_mlp_query(VP(net), C.byref(info)))
    return info


def pc_mlp_set_params(net: int, params) -> None:
    p = _arr(params, np.float32)
    _check(lib().pc_mlp_set_params(VP(net), _ptr(p, C.c_float), p.size))


def pc_mlp_get_params(net: int) -> np.ndarray:
    p = np.zeros(pc_mlp_query(net).n_params, np.float32)
    _check(lib().pc_mlp_get_params(VP(net), _ptr(p, C.c_float), p.size))
    return p


def pc_mlp_forward(net: int, d_x: int, n: int, d_y: int) -> None:
    _check(lib().pc_mlp_forward(VP(net), VP(d_x), n, VP(d_y)))


def pc_mlp_set_gemm(net: int, kind: int) -> None:
    """MLP_GEMM_AUTO (tcgen05 forward products where available) or
    MLP_GEMM_MMA_SYNC (the warp-level kernel for every product)."""
    _check(lib().pc_mlp_set_gemm(VP(net), int(kind)))


def pc_mlp_gemm_info(net: int) -> bool:
    """True when the forward products run on the tcgen05 tensor cores."""
    v = C.c_int32(0)
    _check(lib().pc_mlp_gemm_info(VP(net), C.byref(v)))
    return bool(v.value)


def pc_mlp_gradients(net: int, d_x: int, d_t: int, w, n: int, d_grads: Optional[int] = None) -> float:
    wv = _arr(w, np.float32)
    loss = DBL()
    _check(lib().pc_mlp_gradients(VP(net), VP(d_x), VP(d_t), _ptr(wv, C.c_float), n,
                                  VP(d_grads) if d_grads else None, C.byref(loss)))
    return loss.value


def pc_mlp_train(net: int, d_x: int, d_t: int, n_data: int, w, batch: int, steps: int, lr: float,
                 seed: int) -> float:
    wv = _arr(w, np.float32)
    loss = DBL()
    _check(lib().pc_mlp_train(VP(net), VP(d_x), VP(d_t), n_data, _ptr(wv, C.c_float), batch, steps,
                              float(lr), int(seed), C.byref(loss)))
    return loss.value


def pc_cv_grid(model: int, grid: int, width_sd: float, ref=(1.0, 1.0, 1.0), call_level: float = 1.0,
               ki_level: float = 0.6, coupon: float = 0.05) -> CvDesc:
    """A control-variate description with table axes from the model."""
    desc = CvDesc()
    _check(lib().pc_cv_grid(VP(model), int(grid), float(width_sd), C.byref(desc)))
    for i in range(3):
        desc.ref[i] = float(ref[i]) if i < len(ref) else 1.0
    desc.call_level, desc.ki_level, desc.coupon = float(call_level), float(ki_level), float(coupon)
    return desc


def pc_cv_labels(prices, spots, bump: float, width: int) -> np.ndarray:
    """Labels [n, width] (float32): price, central-difference hedge ratios, zeros."""
    p = _arr(prices, np.float64)
    S = _arr(spots, np.float64)
    n, d = S.shape
    if p.size != (2 * d + 1) * n:
        raise ValueError(f"prices: need {(2 * d + 1) * n} values ([2d + 1, n]), got {p.size}")
    out = np.zeros((n, width), np.float32)
    _check(lib().pc_cv_labels(n, d, _ptr(p, C.c_double), _ptr(S, C.c_double), float(bump), int(width),
                              _ptr(out, C.c_float)))
    return out


def pc_cv_table_size(desc: CvDesc) -> int:
    n = SZ(0)
    _check(lib().pc_cv_table_size(C.byref(desc), C.byref(n)))
    return n.value


def pc_cv_tables(net: int, model: int, desc: CvDesc, d_tables: int, cap_floats: int) -> None:
    _check(lib().pc_cv_tables(VP(net), VP(model), C.byref(desc), VP(d_tables), int(cap_floats)))


def pc_cv_tables_async(net: int, model: int, desc: CvDesc, d_tables: int, cap_floats: int) -> None:
    """pc_cv_tables without the wait: delta0 stays on the device, after the
    tables (cap_floats >= table size + 4)."""
    _check(lib().pc_cv_tables_async(VP(net), VP(model), C.byref(desc), VP(d_tables), int(cap_floats)))


def pc_price_cv(model: int, contract: int, desc: CvDesc, d_tables: int, n_paths: int, seed: int):
    """(price, se) of the control-variate estimate Y = X - beta M - beta2 M2,
    then (price, se) of the plain estimate on the same paths."""
    out = np.zeros(4)
    _check(lib().pc_price_cv(VP(model), VP(contract), C.byref(desc), VP(d_tables), int(n_paths), int(seed),
                             _ptr(out, C.c_double)))
    return (out[0], out[1]), (out[2], out[3])


def pc_cv_beta(model: int, contract: int, desc: CvDesc, d_tables: int, n_paths: int, seed: int):
    """Variance-minimising (beta, beta2) measured on a pilot run."""
    out = np.zeros(2)
    _check(lib().pc_cv_beta(VP(model), VP(contract), C.byref(desc), VP(d_tables), int(n_paths), int(seed),
                            _ptr(out, C.c_double)))
    return float(out[0]), float(out[1])


def pc_debug_cv_paths(model: int, contract: int, desc: CvDesc, d_tables: int, n_paths: int, seed: int,
                      d_xm: int) -> None:
    _check(lib().pc_debug_cv_paths(VP(model), VP(contract), C.byref(desc), VP(d_tables), int(n_paths),
                                   int(seed), VP(d_xm)))


def pc_greeks(model: int, contract: int, n_paths: int, seed: int, d: int):
    """Returns (price, delta[d], vega[d], se[1 + 2d])."""
    p = DBL()
    de, ve, se = np.zeros(d), np.zeros(d), np.zeros(1 + 2 * d)
    _check(lib().pc_greeks(VP(model), VP(contract), n_paths, seed, C.byref(p),
                           _ptr(de, C.c_double), _ptr(ve, C.c_double), _ptr(se, C.c_double)))
    return p.value, de, ve, se


def pc_greeks_adjoint(model: int, contract: int, n_paths: int, seed: int, d: int):
    """(price, delta[d], vega[d], se[1+2d]) from one adjoint launch."""
    price = DBL()
    delta, vega, se = np.zeros(d), np.zeros(d), np.zeros(1 + 2 * d)
    _check(lib().pc_greeks_adjoint(VP(model), VP(contract), n_paths, seed, C.byref(price),
                                   _ptr(delta, C.c_double), _ptr(vega, C.c_double), _ptr(se, C.c_double)))
    return price.value, delta, vega, se


def pc_greeks_adjoint_async(model: int, contract: int, n_paths: int, path_offset: int, seed: int,
                            stream: int, d_out: int) -> None:
    _check(lib().pc_greeks_adjoint_async(VP(model), VP(contract), n_paths, path_offset, seed, stream,
                                         VP(d_out)))


def pc_debug_adjoint_paths(model: int, contract: int, n_paths: int, path_offset: int, seed: int,
                           d_out: int, d_paths: int) -> None:
    _check(lib().pc_debug_adjoint_paths(VP(model), VP(contract), n_paths, path_offset, seed,
                                        VP(d_out), VP(d_paths)))


def pc_debug_philox(ctx: int, d_ctr: int, key0: int, key1: int, d_out: int, n: int) -> None:
    _check(lib().pc_debug_philox(VP(ctx), VP(d_ctr), key0, key1, VP(d_out), n))


def pc_debug_greeks_paths(model: int, contract: int, n_paths: int, path_offset: int, seed: int,
                          underlying: int, d_out: int, d_paths: int) -> None:
    _check(lib().pc_debug_greeks_paths(VP(model), VP(contract), n_paths, path_offset, seed,
                                       underlying, VP(d_out), VP(d_paths)))


def pc_debug_paths(model: int, n_paths: int, path_offset: int, seed: int, stream_id: int,
                   d_S: int) -> None:
    _check(lib().pc_debug_paths(VP(model), n_paths, path_offset, seed, stream_id, VP(d_S)))


def pc_debug_program(words, consts, tparams=(), p1: int = 0, p2: int = 1):
    """Executable form of a program: (uint32 [n_insn, 4], float32 pool)."""
    w, k, t = _arr(words, np.uint32), _arr(consts, np.float64), _arr(tparams, np.int32)
    n, npool = SZ(0), SZ(0)
    lib().pc_debug_program(_ptr(w, C.c_uint32), w.size, _ptr(k, C.c_double), k.size,
                           _ptr(t, C.c_int32), t.size, p1, p2, None, 0, C.byref(n), C.byref(npool))
    out = np.zeros(4 * n.value + npool.value + 1, np.uint32)
    _check(lib().pc_debug_program(_ptr(w, C.c_uint32), w.size, _ptr(k, C.c_double), k.size,
                                  _ptr(t, C.c_int32), t.size, p1, p2,
                                  out.ctypes.data_as(C.POINTER(C.c_uint32)), out.size,
                                  C.byref(n), C.byref(npool)))
    code = out[:4 * n.value].reshape(n.value, 4)
    pool = out[4 * n.value:4 * n.value + npool.value].view(np.float32)
    return code, pool


def pc_debug_bridge(S0, sigma, corr, r, days, t_now=0, history=None, hist_days=None):
    """(date_ops int32 [n+2], ops uint32 [n_ops, 6]) of the model these
    arguments describe (host only)."""
    desc, _keep = _model_desc(S0, sigma, corr, r, days, t_now, history, hist_days)
    n = SZ(0)
    lib().pc_debug_bridge(C.byref(desc), None, None, 0, C.byref(n))
    dops = np.zeros(len(days) + 2, np.int32)
    ops = np.zeros((max(n.value, 1), 6), np.uint32)
    _check(lib().pc_debug_bridge(C.byref(desc), dops.ctypes.data_as(C.POINTER(C.c_int32)),
                                 ops.ctypes.data_as(C.POINTER(C.c_uint32)), ops.shape[0],
                                 C.byref(n)))
    return dops, ops[:n.value]
