"""The no-allocation entry point gb_dtrsm_mixed_noalloc, through the C-ABI.

It exists for callers that must not allocate device memory (their memory is
owned by another allocator, or the allocator may not be called where they
run); it works from a fixed scratch array inside the library.  Checked here:
two calls in a row on different problems (so the second sees the first's
leftovers in the shared scratch) each match gb_dtrsm_mixed on the same
inputs within the mixed path's 1e-10 tolerance (and the FP64 oracle), and a
problem larger than the scratch is refused without touching B.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_2305_19917_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19917_gb300 import build
    build.build()


def _run(fn_name, side, uplo, trans, diag, alpha, A, B):
    import torch
    from paper_2305_19917_gb300 import api
    Ad = api.to_device_colmajor(A, torch.float64)
    Bd = api.to_device_colmajor(B, torch.float64)
    m, n = B.shape
    fn = getattr(api, fn_name)
    st, it, est = fn(side, uplo, trans, diag, m, n, alpha, Ad.data_ptr(), Ad.stride(1) if Ad.shape[1] > 1 else m,
                     Bd.data_ptr(), Bd.stride(1) if n > 1 else m, 1e-11, api.PREC_BF16, 30,
                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, Bd.cpu().numpy()


@pytest.mark.parametrize("first,second", [
    ((0, 0, 0, 0, 300, 170, 1.5, 11), (1, 1, 1, 1, 200, 256, -0.5, 12)),
])
def test_noalloc_matches_allocating_entry_twice(first, second):
    for side, uplo, trans, diag, m, n, alpha, seed in (first, second):
        A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed)
        st_ref, X_ref = _run("gb_dtrsm_mixed", side, uplo, trans, diag, alpha, A, B)
        st, X = _run("gb_dtrsm_mixed_noalloc", side, uplo, trans, diag, alpha, A, B)
        assert st_ref == 0 and st == 0, (st_ref, st)
        assert np.linalg.norm(X - X_ref) <= TOL * np.linalg.norm(X_ref)
        Xo = oracle.dtrsm(side, uplo, trans, diag, alpha, A, B)
        assert np.linalg.norm(X - Xo) <= TOL * np.linalg.norm(Xo)


def test_noalloc_refuses_problems_beyond_its_scratch():
    import torch
    from paper_2305_19917_gb300 import api
    m = n = 1024  # padded work space ~45 MB > 16 MiB
    A, B = inputs.make_problem(0, 0, 0, 0, m, n, seed=1)
    Ad = api.to_device_colmajor(A, torch.float64)
    Bd = api.to_device_colmajor(B, torch.float64)
    st, it, est = api.gb_dtrsm_mixed_noalloc(0, 0, 0, 0, m, n, 1.0, Ad.data_ptr(), m, Bd.data_ptr(), m, 1e-11,
                                             api.PREC_BF16, 30, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == api.STATUS_SCRATCH_TOO_SMALL
    assert np.array_equal(Bd.cpu().numpy(), B)


# The child process below holds no torch: it creates the context and the
# caller's buffers with the CUDA driver API (ctypes), so the only device
# memory that changes hands is what the library itself might take.
# CUDA_MODULE_LOADING=EAGER loads every module of the library (its kernels'
# code and the scratch array) when the library's runtime starts, which the
# first call (alpha = 0, a plain zero fill) does; from then on the device's
# free bytes must not move across the solves.
_COLD_CHILD = r'''
import ctypes, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2305_19917_gb300 import api, inputs

cu = ctypes.CDLL("libcuda.so.1")
def ok(r, what):
    if r != 0:
        raise SystemExit(f"{what} failed: CUresult {r}")
ok(cu.cuInit(0), "cuInit")
dev = ctypes.c_int()
ok(cu.cuDeviceGet(ctypes.byref(dev), 0), "cuDeviceGet")
ctx = ctypes.c_void_p()
ok(cu.cuDevicePrimaryCtxRetain(ctypes.byref(ctx), dev), "cuDevicePrimaryCtxRetain")
ok(cu.cuCtxSetCurrent(ctx), "cuCtxSetCurrent")
cu.cuMemAlloc_v2.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.c_size_t]
cu.cuMemcpyHtoD_v2.argtypes = [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t]
cu.cuMemcpyDtoH_v2.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t]
cu.cuMemGetInfo_v2.argtypes = [ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]

def dalloc(nbytes):
    p = ctypes.c_uint64()
    ok(cu.cuMemAlloc_v2(ctypes.byref(p), nbytes), "cuMemAlloc")
    return p.value

def free_bytes():
    f, t = ctypes.c_size_t(), ctypes.c_size_t()
    ok(cu.cuCtxSynchronize(), "cuCtxSynchronize")
    ok(cu.cuMemGetInfo_v2(ctypes.byref(f), ctypes.byref(t)), "cuMemGetInfo")
    return int(f.value)

problems = [(0, 0, 0, 0, 300, 170, 1.5, 11), (1, 1, 1, 1, 200, 256, -0.5, 12)]
bufs = []
for side, uplo, trans, diag, m, n, alpha, seed in problems:
    A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed)
    A = np.asfortranarray(A); B = np.asfortranarray(B)
    dA, dB = dalloc(A.nbytes), dalloc(B.nbytes)
    ok(cu.cuMemcpyHtoD_v2(dA, A.ctypes.data, A.nbytes), "cuMemcpyHtoD")
    ok(cu.cuMemcpyHtoD_v2(dB, B.ctypes.data, B.nbytes), "cuMemcpyHtoD")
    bufs.append((dA, dB))
dZ = dalloc(64 * 8)

api.lib()
# first library call: alpha = 0 (B := 0, no work space); starts the library's runtime
st0, _, _ = api.gb_dtrsm_mixed_noalloc(0, 0, 0, 0, 8, 8, 0.0, 0, 8, dZ, 8, 1e-11, api.PREC_BF16, 30, 0)
frees = [free_bytes()]
out = {"st0": st0, "runs": []}
for (side, uplo, trans, diag, m, n, alpha, seed), (dA, dB) in zip(problems, bufs):
    k = m if side == 0 else n
    st, it, est = api.gb_dtrsm_mixed_noalloc(side, uplo, trans, diag, m, n, alpha, dA, k, dB, m, 1e-11,
                                             api.PREC_BF16, 30, 0)
    frees.append(free_bytes())
    X = np.empty((m, n), order="F")
    ok(cu.cuMemcpyDtoH_v2(X.ctypes.data, dB, X.nbytes), "cuMemcpyDtoH")
    np.save(sys.argv[2] + f"_{seed}.npy", X)
    out["runs"].append({"st": st, "iters": it, "seed": seed})
out["free"] = frees
print(json.dumps(out))
'''


def test_noalloc_first_call_of_a_cold_process_allocates_nothing(tmp_path):
    """gb_dtrsm_mixed_noalloc as the first library call of a fresh process:
    the device's free memory is the same before and after each of two
    solves, and both match the oracle."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "child.py"
    script.write_text(_COLD_CHILD)
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    r = subprocess.run([sys.executable, str(script), root, str(tmp_path / "X")], capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["st0"] == 0
    assert all(run["st"] == 0 for run in out["runs"]), out
    frees = out["free"]
    assert frees[1] == frees[0] and frees[2] == frees[0], f"free device bytes moved: {frees}"
    for side, uplo, trans, diag, m, n, alpha, seed in ((0, 0, 0, 0, 300, 170, 1.5, 11),
                                                         (1, 1, 1, 1, 200, 256, -0.5, 12)):
        A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed)
        X = np.load(tmp_path / f"X_{seed}.npy")
        Xo = oracle.dtrsm(side, uplo, trans, diag, alpha, A, B)
        assert np.linalg.norm(X - Xo) <= TOL * np.linalg.norm(Xo)
