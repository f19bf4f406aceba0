"""In-tree build of the engine's shared library ``libpc.so`` for sm_103a.

Compiles the CUDA translation units with nvcc
(``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3``) and the host C++
units with g++, in parallel, then links them with the shared CUDA runtime.
Outputs go to ``_build/`` and ``libpc.so`` next to this file (both ignored by
git).  Rebuilds only when a source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import re
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.inc")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


# Device sources the run-time compiler (NVRTC) needs, embedded in the
# library as string literals (pc_jit.cpp includes the generated header).
JIT_HEADERS = ["pc_types.h", "pc_device.cuh", "pc_price.cuh", "pc_eval_state.inc", "pc_ops.inc", "pc_cv_types.h",
               "pc_cv.cuh", "pc_greeks.cuh", "pc_greeks_state.inc", "pc_greeks_ops.inc", "pc_adjoint.cuh",
               "pc_adjoint_state.inc", "pc_adjoint_ops.inc"]


def _op_cases():
    """Case text of each opcode in pc_ops.inc, indexed by the XOp value (the
    enum's order in pc_types.h); X_END takes the default case."""
    with open(os.path.join(CSRC, "pc_types.h")) as f:
        types = f.read()
    e = types[types.index("enum XOp : uint32_t {") + len("enum XOp : uint32_t {"):]
    e = re.sub(r"//[^\n]*", "", e[:e.index("};")])
    names = [x.strip().split("=")[0].strip() for x in e.split(",") if x.strip()]
    with open(os.path.join(CSRC, "pc_ops.inc")) as f:
        lines = f.read().splitlines(keepends=True)
    groups, cur = [], None
    for ln in lines:
        m = re.match(r"^      case (X_\w+):(.*)$", ln, re.S)
        if m or ln.startswith("      default:"):
            if cur is not None and cur[1]:
                groups.append(cur)
                cur = None
            if cur is None:
                cur = ([], [])
            label, rest = (m.group(1), m.group(2)) if m else ("default", ln.split("default:", 1)[1])
            cur[0].append(label)
            if rest.strip():
                cur[1].append("      " + rest.lstrip())
        elif cur is not None:
            cur[1].append(ln)
    if cur is not None:
        groups.append(cur)
    text = {lab: "".join(body) for labels, body in groups for lab in labels}
    return [text.get(n, text["default"]) for n in names]


def _jit_headers() -> None:
    out = os.path.join(BUILD, "pc_jit_headers.inc")
    parts = ["// generated by build.py: device sources for the run-time compiler\n"]
    names, srcs = [], []
    for i, h in enumerate(JIT_HEADERS):
        with open(os.path.join(CSRC, h)) as f:
            text = f.read()
        if ")PCJIT\"" in text:
            raise RuntimeError(f"{h} contains the raw-string delimiter")
        parts.append(f"static const char kJitSrc{i}[] = R\"PCJIT({text})PCJIT\";\n")
        names.append(f'"{h}"')
        srcs.append(f"kJitSrc{i}")
    parts.append(f"static const int kJitHeaderCount = {len(JIT_HEADERS)};\n")
    parts.append("static const char *const kJitHeaderNames[] = {" + ", ".join(names) + "};\n")
    parts.append("static const char *const kJitHeaderSrcs[] = {" + ", ".join(srcs) + "};\n")
    cases = _op_cases()
    for i, c in enumerate(cases):
        parts.append(f"static const char kJitCase{i}[] = R\"PCJIT({c})PCJIT\";\n")
    parts.append(f"static const int kJitCaseCount = {len(cases)};\n")
    parts.append("static const char *const kJitCase[] = {" +
                 ", ".join(f"kJitCase{i}" for i in range(len(cases))) + "};\n")
    text = "".join(parts)
    if not os.path.exists(out) or open(out).read() != text:
        with open(out, "w") as f:
            f.write(text)


def _compile(src: str, cuda: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-I" + BUILD, "-I" + os.path.join(cuda, "include")]
    if src.endswith(".cu"):
        cmd = [os.path.join(cuda, "bin", "nvcc"), *ARCH, "-lineinfo", "-O3", "-std=c++17",
               "-Xcompiler", "-fPIC", "-Xptxas", "-v" if verbose else "-O3", *inc, "-c", src, "-o", obj]
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function", *inc,
               "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libpc.so if needed and return its path."""
    if not force and up_to_date():
        return LIB
    cuda = cuda_home()
    os.makedirs(BUILD, exist_ok=True)
    _jit_headers()
    with concurrent.futures.ThreadPoolExecutor(max_workers=8) as ex:
        objs = list(ex.map(lambda s: _compile(s, cuda, verbose), _sources()))
    tmp = LIB + ".tmp"
    cmd = [os.path.join(cuda, "bin", "nvcc"), *ARCH, "-shared", "-cudart", "shared", "-o", tmp,
           *objs, "-L" + os.path.join(cuda, "lib64"), "-lnvrtc"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
