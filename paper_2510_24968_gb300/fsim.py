"""Python binding of libfsim (include/fsim.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts molecules to
the C structs, passes host arrays or device pointers (torch tensors) through,
and turns return codes into exceptions.  If libfsim.so is missing or cannot be
loaded the import fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfsim.so")

FSIM_OK = 0
FSIM_EINVAL = -1
FSIM_ECUDA = -2
FSIM_ENOCONV = -3
FSIM_EILLCOND = -4
FSIM_EDEVICE_TIMEOUT = -5
FSIM_ENOMEM = -6
FSIM_FP64 = 0
FSIM_MIXED = 1
FSIM_DFLOAT = 2
FSIM_BASIS_SPHERICAL = 1
FSIM_PTR_HOST = 0
FSIM_PTR_DEVICE = 1
FSIM_GUESS_CORE = 0
FSIM_GUESS_DENSITY = 1
FSIM_GUESS_LEARNED = 2

# every symbol declared in include/fsim.h
EXPORTS = ["fsim_basis_create", "fsim_basis_create_ex", "fsim_basis_destroy", "fsim_basis_nbf",
           "fsim_basis_nbf_cart", "fsim_basis_nshell",
           "fsim_basis_pair_counts", "fsim_enuc", "fsim_onee", "fsim_schwarz", "fsim_fock_opts_default",
           "fsim_fock_build", "fsim_fock_build_noalloc", "fsim_j_build", "fsim_autotune", "fsim_set_launch", "fsim_last_quartet_count", "fsim_last_class_times", "fsim_eri_quartets", "fsim_eri_dump",
           "fsim_scf_opts_default", "fsim_scf", "fsim_batch_create", "fsim_batch_fock", "fsim_batch_destroy",
           "fsim_scf_batched", "fsim_guess_layout", "fsim_guess_features", "fsim_guess_targets",
           "fsim_guess_assemble", "fsim_mlp_create", "fsim_mlp_destroy", "fsim_mlp_nparams", "fsim_mlp_params",
           "fsim_mlp_save", "fsim_mlp_load", "fsim_mlp_adam_step", "fsim_mlp_forward", "fsim_mlp_grad", "fsim_mlp_train_step",
           "fsim_last_error"]


class FsimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fsim error {code}: {msg}")
        self.code = code


class fsim_atom(C.Structure):
    _fields_ = [("Z", C.c_int), ("xyz", C.c_double * 3)]


class fsim_shell_desc(C.Structure):
    _fields_ = [("atom", C.c_int), ("l", C.c_int), ("nprim", C.c_int),
                ("alpha", C.POINTER(C.c_double)), ("coef", C.POINTER(C.c_double))]


class fsim_fock_opts(C.Structure):
    _fields_ = [("schwarz_tau", C.c_double), ("precision", C.c_int), ("boys_fp64_T", C.c_double),
                ("ptr_mode", C.c_int), ("stream", C.c_void_p), ("shard", C.c_int), ("nshards", C.c_int),
                ("timing", C.c_int)]


class fsim_scf_opts(C.Structure):
    _fields_ = [("nelec", C.c_int), ("max_iter", C.c_int), ("conv_dE", C.c_double), ("conv_dD", C.c_double),
                ("diis_size", C.c_int), ("guess", C.c_int), ("D0", C.POINTER(C.c_double)),
                ("fock", fsim_fock_opts), ("final_fp64", C.c_int), ("incremental", C.c_int),
                ("guess_model", C.c_char_p), ("dw_screen", C.c_int)]


class fsim_scf_result(C.Structure):
    _fields_ = [("e_total", C.c_double), ("e_elec", C.c_double), ("e_nuc", C.c_double), ("iters", C.c_int),
                ("converged", C.c_int), ("guess_fallback", C.c_int), ("D_out", C.POINTER(C.c_double)),
                ("e_hist", C.POINTER(C.c_double)), ("t_hist", C.POINTER(C.c_double)), ("time_s", C.c_double),
                ("min_s_eig", C.c_double), ("quartets", C.c_longlong), ("fp64_builds", C.c_int),
                ("mixed_builds", C.c_int), ("guess_s", C.c_double), ("mixed_fallback", C.c_int)]


_lib = None


def load():
    """Load libfsim.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfsim.so not built ({LIB_PATH}); run paper_2510_24968_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    dp, ip, vp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p
    L.fsim_basis_create.argtypes = [C.POINTER(fsim_atom), C.c_int, C.POINTER(fsim_shell_desc), C.c_int,
                                    C.POINTER(vp)]
    L.fsim_basis_create_ex.argtypes = [C.POINTER(fsim_atom), C.c_int, C.POINTER(fsim_shell_desc), C.c_int, C.c_int,
                                       C.POINTER(C.c_void_p)]
    L.fsim_basis_nbf_cart.argtypes = [vp]
    L.fsim_basis_destroy.argtypes = [vp]
    L.fsim_basis_destroy.restype = None
    L.fsim_basis_nbf.argtypes = [vp]
    L.fsim_basis_nshell.argtypes = [vp]
    L.fsim_basis_pair_counts.argtypes = [vp, ip]
    L.fsim_enuc.argtypes = [vp, dp]
    L.fsim_onee.argtypes = [vp, C.c_int, vp, C.c_int, vp]
    L.fsim_schwarz.argtypes = [vp, dp]
    L.fsim_fock_opts_default.argtypes = [C.POINTER(fsim_fock_opts)]
    L.fsim_fock_opts_default.restype = None
    L.fsim_fock_build.argtypes = [vp, vp, vp, vp, C.POINTER(fsim_fock_opts)]
    L.fsim_fock_build_noalloc.argtypes = [vp, vp, vp, vp, C.POINTER(fsim_fock_opts)]
    L.fsim_j_build.argtypes = [vp, vp, vp, C.POINTER(fsim_fock_opts)]
    L.fsim_autotune.argtypes = [vp, C.POINTER(fsim_fock_opts), ip, C.POINTER(C.c_float)]
    L.fsim_set_launch.argtypes = [vp, C.POINTER(fsim_fock_opts), ip]
    L.fsim_last_quartet_count.argtypes = [vp]
    L.fsim_last_quartet_count.restype = C.c_longlong
    L.fsim_last_class_times.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_longlong), ip]
    L.fsim_eri_quartets.argtypes = [vp, C.c_int, ip, dp, C.c_int]
    L.fsim_eri_dump.argtypes = [vp, dp, C.c_int]
    L.fsim_scf_opts_default.argtypes = [C.POINTER(fsim_scf_opts)]
    L.fsim_scf_opts_default.restype = None
    L.fsim_scf.argtypes = [vp, C.POINTER(fsim_scf_opts), C.POINTER(fsim_scf_result)]
    L.fsim_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(fsim_fock_opts), C.POINTER(vp),
                                    C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]
    L.fsim_batch_fock.argtypes = [vp, C.c_int, ip, C.c_int]
    L.fsim_batch_destroy.argtypes = [vp]
    L.fsim_batch_destroy.restype = None
    L.fsim_scf_batched.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(fsim_scf_opts), C.POINTER(fsim_scf_result)]
    fp = C.POINTER(C.c_float)
    L.fsim_guess_layout.argtypes = [vp, ip, ip, ip]
    L.fsim_guess_features.argtypes = [vp, fp]
    L.fsim_guess_targets.argtypes = [vp, dp, fp, fp]
    L.fsim_guess_assemble.argtypes = [vp, vp, vp, vp]
    L.fsim_mlp_create.argtypes = [C.c_int, C.c_int, C.c_int, fp, C.POINTER(vp)]
    L.fsim_mlp_destroy.argtypes = [vp]
    L.fsim_mlp_destroy.restype = None
    L.fsim_mlp_nparams.argtypes = [vp]
    L.fsim_mlp_nparams.restype = C.c_longlong
    L.fsim_mlp_params.argtypes = [vp, fp, fp]
    L.fsim_mlp_save.argtypes = [vp, C.c_char_p]
    L.fsim_mlp_adam_step.argtypes = [vp, C.POINTER(C.c_float), C.c_float, vp]
    L.fsim_mlp_load.argtypes = [C.c_char_p, C.POINTER(vp)]
    L.fsim_mlp_forward.argtypes = [vp, vp, vp, C.c_int, C.c_int, vp]
    L.fsim_mlp_grad.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int, fp, fp, vp]
    L.fsim_mlp_train_step.argtypes = [vp, vp, vp, vp, C.c_int, C.c_float, fp, vp]
    L.fsim_last_error.restype = C.c_char_p
    _lib = L
    return L


def _check(rc, allow=()):
    if rc != FSIM_OK and rc not in allow:
        raise FsimError(rc, load().fsim_last_error().decode())
    return rc


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ptr_of(x):
    """(pointer, mode) for a numpy array (host) or a CUDA torch tensor (device)."""
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float64 and x.flags.c_contiguous
        return C.c_void_p(x.ctypes.data), FSIM_PTR_HOST
    # torch tensor
    assert x.dtype.__str__() == "torch.float64" and x.is_contiguous()
    return C.c_void_p(x.data_ptr()), (FSIM_PTR_DEVICE if x.is_cuda else FSIM_PTR_HOST)


def fsim_fock_opts_default() -> fsim_fock_opts:
    o = fsim_fock_opts()
    load().fsim_fock_opts_default(C.byref(o))
    return o


def fsim_scf_opts_default() -> fsim_scf_opts:
    o = fsim_scf_opts()
    load().fsim_scf_opts_default(C.byref(o))
    return o


class Basis:
    """Owns an fsim_basis handle built from a fsim_synth.Molecule."""

    def __init__(self, mol, spherical=False):
        L = load()
        a = mol.arrays()
        atoms = (fsim_atom * mol.natom)()
        for i in range(mol.natom):
            atoms[i].Z = int(a["Z"][i])
            for x in range(3):
                atoms[i].xyz[x] = float(a["xyz"][i, x])
        self._keep = []
        shells = (fsim_shell_desc * mol.nshell)()
        for s, sh in enumerate(mol.shells):
            al = np.array(sh.alpha, dtype=np.float64)
            co = np.array(sh.coef, dtype=np.float64)
            self._keep += [al, co]
            shells[s].atom, shells[s].l, shells[s].nprim = sh.atom, sh.l, len(sh.alpha)
            shells[s].alpha, shells[s].coef = _dptr(al), _dptr(co)
        h = C.c_void_p()
        _check(L.fsim_basis_create_ex(atoms, mol.natom, shells, mol.nshell, FSIM_BASIS_SPHERICAL if spherical else 0,
                                      C.byref(h)))
        self.h = h
        self.mol = mol
        self.spherical = bool(spherical)
        self.nbf = L.fsim_basis_nbf(h)
        self.nbf_cart = L.fsim_basis_nbf_cart(h)
        self.nshell = L.fsim_basis_nshell(h)

    def close(self):
        if getattr(self, "h", None):
            load().fsim_basis_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pair_counts(self):
        c = (C.c_int * 6)()
        _check(load().fsim_basis_pair_counts(self.h, c))
        return list(c)

    def enuc(self) -> float:
        e = C.c_double()
        _check(load().fsim_enuc(self.h, C.byref(e)))
        return e.value

    def onee(self, which: str, out=None, stream=None):
        code = {"S": 0, "T": 1, "V": 2}[which]
        if out is None:
            out = np.zeros((self.nbf, self.nbf))
        p, mode = _ptr_of(out)
        _check(load().fsim_onee(self.h, code, p, mode, C.c_void_p(stream or 0)))
        return out

    def schwarz(self) -> np.ndarray:
        Q = np.zeros((self.nshell, self.nshell))
        _check(load().fsim_schwarz(self.h, _dptr(Q)))
        return Q

    def fock_build(self, D, J=None, K=None, tau=1e-10, precision=FSIM_FP64, stream=None,
                   shard=0, nshards=1, boys_fp64_T=0.0, timing=False):
        """J, K for density D (numpy -> host mode; CUDA torch tensors -> device mode)."""
        if J is None:
            J = np.zeros((self.nbf, self.nbf)) if isinstance(D, np.ndarray) else D.new_zeros(D.shape)
        if K is None:
            K = np.zeros((self.nbf, self.nbf)) if isinstance(D, np.ndarray) else D.new_zeros(D.shape)
        o = fsim_fock_opts_default()
        o.schwarz_tau, o.precision, o.shard, o.nshards = tau, precision, shard, nshards
        o.boys_fp64_T, o.timing = boys_fp64_T, int(timing)
        pD, mode = _ptr_of(D)
        pJ, _ = _ptr_of(J)
        pK, _ = _ptr_of(K)
        o.ptr_mode = mode
        o.stream = stream or 0
        _check(load().fsim_fock_build(self.h, pD, pJ, pK, C.byref(o)))
        return J, K

    def j_build(self, D, J=None, tau=1e-10, precision=FSIM_FP64, stream=None, shard=0, nshards=1,
                boys_fp64_T=0.0):
        """J alone for density D by the Hermite-space J-engine (numpy -> host mode; CUDA torch
        tensors -> device mode)."""
        if J is None:
            J = np.zeros((self.nbf, self.nbf)) if isinstance(D, np.ndarray) else D.new_zeros(D.shape)
        o = fsim_fock_opts_default()
        o.schwarz_tau, o.precision, o.shard, o.nshards = tau, precision, shard, nshards
        o.boys_fp64_T = boys_fp64_T
        pD, mode = _ptr_of(D)
        pJ, _ = _ptr_of(J)
        o.ptr_mode = mode
        o.stream = stream or 0
        _check(load().fsim_j_build(self.h, pD, pJ, C.byref(o)))
        return J

    def autotune(self, tau=1e-10, precision=FSIM_MIXED, stream=None, shard=0, nshards=1):
        """Tune the launch shape of every class pair; returns {(X, Y): (choice, ms)}."""
        o = fsim_fock_opts_default()
        o.schwarz_tau, o.precision, o.shard, o.nshards = tau, precision, shard, nshards
        o.stream = stream or 0
        ch = (C.c_int * 36)()
        ms = (C.c_float * 36)()
        _check(load().fsim_autotune(self.h, C.byref(o), ch, ms))
        return {(i // 6, i % 6): (ch[i], ms[i]) for i in range(36) if ch[i] != 0}

    def set_launch(self, choices, tau=1e-10, precision=FSIM_MIXED, shard=0, nshards=1):
        """Launch shapes {(X, Y): choice} in fsim_autotune's encoding (e.g. a saved tuning)."""
        o = fsim_fock_opts_default()
        o.schwarz_tau, o.precision, o.shard, o.nshards = tau, precision, shard, nshards
        ch = (C.c_int * 36)()
        for (x, y), c in choices.items():
            ch[x * 6 + y] = int(c)
        _check(load().fsim_set_launch(self.h, C.byref(o), ch))

    def last_quartet_count(self) -> int:
        return load().fsim_last_quartet_count(self.h)

    def last_class_times(self):
        """({(X, Y): ms}, {(X, Y): quartets}, kernels launched) of the last build."""
        ms = (C.c_float * 36)()
        q = (C.c_longlong * 36)()
        n = C.c_int()
        _check(load().fsim_last_class_times(self.h, ms, q, C.byref(n)))
        times = {(i // 6, i % 6): ms[i] for i in range(36) if ms[i] >= 0}
        quart = {(i // 6, i % 6): q[i] for i in range(36) if i // 6 >= i % 6}
        return times, quart, n.value

    def eri_quartets(self, quartets) -> list:
        q = np.ascontiguousarray(np.asarray(quartets, dtype=np.int32).reshape(-1, 4))
        ls = [s.l for s in self.mol.shells]
        sizes = [int(np.prod([(ls[s] + 1) * (ls[s] + 2) // 2 for s in row])) for row in q]
        out = np.zeros(sum(sizes))
        _check(load().fsim_eri_quartets(self.h, len(q), q.ctypes.data_as(C.POINTER(C.c_int)), _dptr(out),
                                        FSIM_FP64))
        blocks, off = [], 0
        for row, sz in zip(q, sizes):
            shp = [(ls[s] + 1) * (ls[s] + 2) // 2 for s in row]
            blocks.append(out[off:off + sz].reshape(shp))
            off += sz
        return blocks

    def eri_dump(self) -> np.ndarray:
        """All Cartesian ERIs (nbf_cart^4), also for spherical bases."""
        N = self.nbf_cart
        g = np.zeros(N ** 4)
        _check(load().fsim_eri_dump(self.h, _dptr(g), FSIM_FP64))
        return g.reshape(N, N, N, N)

    def scf(self, nelec=None, precision=FSIM_FP64, tau=1e-10, max_iter=100, conv_dE=1e-10, conv_dD=1e-7,
            diis_size=8, D0=None, final_fp64=2, incremental=True, stream=None, want_density=False,
            guess_model=None, dw_screen=False):
        o = fsim_scf_opts_default()
        o.nelec = self.mol.nelec if nelec is None else nelec
        o.max_iter, o.conv_dE, o.conv_dD, o.diis_size = max_iter, conv_dE, conv_dD, diis_size
        o.fock.schwarz_tau, o.fock.precision = tau, precision
        o.fock.stream = stream or 0
        o.final_fp64, o.incremental = int(final_fp64), int(incremental)
        o.dw_screen = int(dw_screen)
        keep = []
        if D0 is not None:
            d0 = np.ascontiguousarray(D0, dtype=np.float64)
            keep.append(d0)
            o.guess, o.D0 = FSIM_GUESS_DENSITY, _dptr(d0)
        elif guess_model is not None:
            path = os.fsencode(guess_model)
            keep.append(path)
            o.guess, o.guess_model = FSIM_GUESS_LEARNED, path
        r = fsim_scf_result()
        eh = np.full(max_iter, np.nan)
        th = np.full(max_iter, np.nan)
        r.e_hist, r.t_hist = _dptr(eh), _dptr(th)
        Dout = None
        if want_density:
            Dout = np.zeros((self.nbf, self.nbf))
            r.D_out = _dptr(Dout)
        rc = _check(load().fsim_scf(self.h, C.byref(o), C.byref(r)), allow=(FSIM_ENOCONV,))
        n = r.iters
        return {"e_total": r.e_total, "e_elec": r.e_elec, "e_nuc": r.e_nuc, "iters": n,
                "converged": bool(r.converged), "rc": rc, "time_s": r.time_s, "min_s_eig": r.min_s_eig,
                "quartets": r.quartets, "fp64_builds": r.fp64_builds, "mixed_builds": r.mixed_builds,
                "energies": eh[:n].copy(), "times": th[:n].copy(), "D": Dout,
                "guess_fallback": bool(r.guess_fallback), "guess_s": r.guess_s,
                "mixed_fallback": bool(r.mixed_fallback)}


class Batch:
    """A set of bases bound to device buffers D[m] -> J[m], K[m] (CUDA torch tensors)."""

    def __init__(self, bases, D, J, K, tau=1e-10, stream=None):
        L = load()
        n = len(bases)
        self.bases, self._keep = bases, (D, J, K)
        hb = (C.c_void_p * n)(*[b.h.value for b in bases])
        hd = (C.c_void_p * n)(*[d.data_ptr() for d in D])
        hj = (C.c_void_p * n)(*[x.data_ptr() for x in J])
        hk = (C.c_void_p * n)(*[x.data_ptr() for x in K])
        o = fsim_fock_opts_default()
        o.schwarz_tau, o.ptr_mode, o.stream = tau, FSIM_PTR_DEVICE, stream or 0
        h = C.c_void_p()
        _check(L.fsim_batch_create(hb, n, C.byref(o), hd, hj, hk, C.byref(h)))
        self.h = h

    def fock(self, precision=FSIM_MIXED, active=None, use_graph=True):
        act = None if active is None else (C.c_int * len(self.bases))(*[int(a) for a in active])
        _check(load().fsim_batch_fock(self.h, precision, act, int(use_graph)))

    def close(self):
        if getattr(self, "h", None):
            load().fsim_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def scf_batched(bases, precision=FSIM_MIXED, tau=1e-10, max_iter=100, conv_dE=1e-10, conv_dD=1e-7, diis_size=8,
                final_fp64=True, incremental=True, stream=None, want_density=False, dw_screen=False):
    """Lockstep RHF of many molecules; returns a list of per-molecule dicts."""
    n = len(bases)
    o = fsim_scf_opts_default()
    o.nelec = 0
    o.max_iter, o.conv_dE, o.conv_dD, o.diis_size = max_iter, conv_dE, conv_dD, diis_size
    o.fock.schwarz_tau, o.fock.precision = tau, precision
    o.fock.stream = stream or 0
    o.final_fp64, o.incremental = int(final_fp64), int(incremental)
    o.dw_screen = int(dw_screen)
    res = (fsim_scf_result * n)()
    hist = [np.full(max_iter, np.nan) for _ in range(n)]
    thist = [np.full(max_iter, np.nan) for _ in range(n)]
    for r, h, t in zip(res, hist, thist):
        r.e_hist, r.t_hist = _dptr(h), _dptr(t)
    dens = [np.zeros((b.nbf, b.nbf)) for b in bases] if want_density else [None] * n
    if want_density:
        for r, d in zip(res, dens):
            r.D_out = _dptr(d)
    hb = (C.c_void_p * n)(*[b.h.value for b in bases])
    rc = _check(load().fsim_scf_batched(hb, n, C.byref(o), res), allow=(FSIM_ENOCONV,))
    return [{"e_total": r.e_total, "iters": r.iters, "converged": bool(r.converged), "time_s": r.time_s,
             "fp64_builds": r.fp64_builds, "mixed_builds": r.mixed_builds, "rc": rc,
             "mixed_fallback": bool(r.mixed_fallback), "min_s_eig": r.min_s_eig,
             "energies": h[:r.iters].copy(), "times": t[:r.iters].copy(), "D": d}
            for r, h, t, d in zip(res, hist, thist, dens)]
