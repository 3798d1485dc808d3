"""fsim_fock_build_noalloc: the Fock build for callers that cannot allocate
device memory while they run (its scratch is a fixed device array inside the
library).  Called through the C-ABI, its J and K must match fsim_fock_build's
within the parity tolerances of the other tests, on two calls in a row (the
shared scratch keeps the previous call's contents, so the second call checks
that it is cleared).  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from fsim_synth import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_24968_gb300.build import build
    build()
    from paper_2510_24968_gb300 import fsim
    return fsim


def _opts(fsim, precision, tau=1e-10):
    o = fsim.fsim_fock_opts_default()
    o.schwarz_tau, o.precision, o.ptr_mode = tau, precision, fsim.FSIM_PTR_DEVICE
    o.stream = torch.cuda.current_stream().cuda_stream
    return o


@pytest.mark.parametrize("prec_name,tol_rel", [("FSIM_FP64", None), ("FSIM_MIXED", 1e-11)])
def test_noalloc_matches_fock_build_twice(lib, prec_name, tol_rel):
    # both entry points run the same kernels on the same plan, so they differ only
    # by the order of the FP64 atomic additions; the second call takes another D,
    # so a stale copy of the first call's density (the FP32 copy in the shared
    # scratch) or uncleared accumulators would show
    fsim = lib
    prec = getattr(fsim, prec_name)
    gb = fsim.Basis(workload("water8"))
    L = fsim.load()
    rng = np.random.default_rng(11)
    Ds = []
    for _ in range(2):
        D = torch.from_numpy(rng.standard_normal((gb.nbf, gb.nbf)) * 0.1).cuda()
        Ds.append((D + D.T).contiguous())
    o = _opts(fsim, prec)
    # set-up with the allocating entry point (Schwarz bounds, screening plan) and the reference results
    refs = []
    for D in Ds:
        Jr, Kr = torch.zeros_like(D), torch.zeros_like(D)
        assert L.fsim_fock_build(gb.h, C.c_void_p(D.data_ptr()), C.c_void_p(Jr.data_ptr()),
                                 C.c_void_p(Kr.data_ptr()), C.byref(o)) == 0
        refs.append((Jr, Kr))
    nq = L.fsim_last_quartet_count(gb.h)
    for call, (D, (Jr, Kr)) in enumerate(zip(Ds, refs)):
        J, K = torch.full_like(D, np.nan), torch.full_like(D, np.nan)
        rc = L.fsim_fock_build_noalloc(gb.h, C.c_void_p(D.data_ptr()), C.c_void_p(J.data_ptr()),
                                       C.c_void_p(K.data_ptr()), C.byref(o))
        assert rc == 0, L.fsim_last_error()
        torch.cuda.synchronize()
        assert L.fsim_last_quartet_count(gb.h) == nq
        dj = torch.abs(J - Jr).max().item()
        dk = torch.abs(K - Kr).max().item()
        if tol_rel is None:
            assert dj < 1e-10 and dk < 1e-10, (call, dj, dk)
        else:
            s = max(torch.abs(Jr).max().item(), torch.abs(Kr).max().item())
            assert dj < tol_rel * s and dk < tol_rel * s, (call, dj, dk)


def test_noalloc_rejects_what_it_cannot_serve(lib):
    fsim = lib
    L = fsim.load()

    def call(gb, o, Dm):
        return L.fsim_fock_build_noalloc(gb.h, C.c_void_p(Dm.data_ptr()), C.c_void_p(Dm.data_ptr()),
                                         C.c_void_p(Dm.data_ptr()), C.byref(o))

    # a fresh basis has no Schwarz bounds yet: refused without launching anything
    gb = fsim.Basis(workload("water"))
    D = torch.zeros((gb.nbf, gb.nbf), dtype=torch.float64, device="cuda")
    o = _opts(fsim, fsim.FSIM_FP64, tau=1e-10)
    assert call(gb, o, D) == fsim.FSIM_EINVAL and b"Schwarz" in L.fsim_last_error()
    # set-up for tau 1e-10 only: a call with tau 1e-7 has no screening plan
    J, K = torch.zeros_like(D), torch.zeros_like(D)
    assert L.fsim_fock_build(gb.h, C.c_void_p(D.data_ptr()), C.c_void_p(J.data_ptr()),
                             C.c_void_p(K.data_ptr()), C.byref(o)) == 0
    o7 = _opts(fsim, fsim.FSIM_FP64, tau=1e-7)
    assert call(gb, o7, D) == fsim.FSIM_EINVAL and b"screening plan" in L.fsim_last_error()
    # the double-float precision needs allocated per-basis copies
    od = _opts(fsim, fsim.FSIM_DFLOAT, tau=1e-10)
    assert call(gb, od, D) == fsim.FSIM_EINVAL and b"precision" in L.fsim_last_error()
    # more basis functions than the fixed scratch holds
    big = fsim.Basis(workload("cloud30"))
    assert big.nbf > 512
    Db = torch.zeros((big.nbf, big.nbf), dtype=torch.float64, device="cuda")
    assert call(big, o, Db) == fsim.FSIM_EINVAL and b"capacity" in L.fsim_last_error()
