"""Device-side generation of :func:`synth.varcoef` systems.

``libsynthgen.so`` (``synth/csrc/synth_gen.cu``) draws the same SplitMix64
streams as the host generator and forms the coefficients with the host's
operations in the same order, so a system generated on the device equals
the host one bit for bit in its coefficients (b may differ by one unit in
the last place in rare cells: log, sqrt and cos come from the device's math
library).  Used where many or large systems are needed on the GPU (request
streams, full-size meshes) and host generation would dominate.  It holds no
solver arithmetic.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

from . import DIRS, STREAM_COEF, STREAM_RHS, stream_key

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "synth_gen.cu")
LIB = os.path.join(HERE, "libsynthgen.so")
_lib = None


def build(force=False):
    """Compile libsynthgen.so for sm_103a (only when the source is newer)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    nvcc = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        nvcc = "nvcc"
    tmp = LIB + ".tmp"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
                    "-Xcompiler", "-fPIC", "-shared", "-o", tmp, SRC], check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libsynthgen.so is not built (run synth.device.build())")
        _lib = C.CDLL(LIB)
        _lib.synth_varcoef_device.restype = C.c_int
        _lib.synth_varcoef_device.argtypes = [C.c_longlong, C.c_uint64, C.c_uint64] + \
            [C.c_void_p] * 10
    return _lib


def varcoef(nx, ny, nz, seed, device, b_dtype="f64"):
    """``(coef, b)`` of ``synth.varcoef(nx, ny, nz, seed)`` (float32 raw values)
    as CUDA tensors on ``device``; b as float64 (holding the float32 values)
    or float32.  Generated on the current torch stream of that device."""
    import torch
    n = nx * ny * nz
    coef = {k: torch.empty(n, dtype=torch.float32, device=device) for k in DIRS + ("diag",)}
    b = torch.empty(n, dtype=torch.float64 if b_dtype == "f64" else torch.float32, device=device)
    st = torch.cuda.current_stream(device).cuda_stream
    rc = lib().synth_varcoef_device(
        n, int(stream_key(seed, STREAM_COEF)), int(stream_key(seed, STREAM_RHS)),
        *[coef[k].data_ptr() for k in DIRS], coef["diag"].data_ptr(),
        b.data_ptr() if b_dtype != "f64" else None, b.data_ptr() if b_dtype == "f64" else None,
        st)
    if rc != 0:
        raise RuntimeError("synth_varcoef_device failed (cudaError %d)" % rc)
    return coef, b
