"""ctypes front end of the C oracle (fsim_oracle.c).

TEST INFRASTRUCTURE ONLY (see the package docstring).  ``build()`` compiles
the C source with the host compiler; nothing here touches a GPU.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsim_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, -O2, OpenMP) if missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_boys.restype = C.c_double
            L.orc_boys.argtypes = [C.c_int, C.c_double]
            L.orc_hermite_E.restype = C.c_double
            L.orc_hermite_E.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]
            L.orc_hermite_R.restype = C.c_double
            L.orc_hermite_R.argtypes = [C.c_int] * 4 + [C.c_double] * 4
            L.orc_basis_create.restype = C.c_void_p
            L.orc_basis_create.argtypes = [C.c_int, _ip, _dp, C.c_int, _ip, _ip, _ip, _dp, _dp]
            L.orc_basis_destroy.argtypes = [C.c_void_p]
            L.orc_basis_nbf.restype = C.c_int
            L.orc_basis_nbf.argtypes = [C.c_void_p]
            L.orc_onee.argtypes = [C.c_void_p, C.c_int, _dp]
            L.orc_enuc.restype = C.c_double
            L.orc_enuc.argtypes = [C.c_void_p]
            L.orc_eri_shell_quartet.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, _dp]
            L.orc_eri_full.argtypes = [C.c_void_p, _dp]
            L.orc_eri_quartet_list.argtypes = [C.c_void_p, C.c_int, _ip, C.POINTER(C.c_longlong), _dp]
            L.orc_schwarz.argtypes = [C.c_void_p, _dp]
            L.orc_jk.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_double, C.c_int,
                                 C.POINTER(C.c_longlong)]
            L.orc_jk_sample.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_double, C.c_int,
                                        C.POINTER(C.c_longlong), C.c_int]
            L.orc_jk_shard.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_double, C.c_int,
                                       C.POINTER(C.c_longlong), C.c_int, C.c_int]
            L.orc_jk_block.argtypes = [C.c_void_p, _dp, C.c_int, C.c_int, _dp, _dp, C.c_double, _dp]
            L.orc_jacobi_eigh.restype = C.c_int
            L.orc_jacobi_eigh.argtypes = [C.c_int, _dp, _dp, _dp]
            _lib = L
    return _lib


def boys(n: int, T: float) -> float:
    """F_n(T) = int_0^1 exp(-T t^2) t^(2n) dt."""
    return lib().orc_boys(int(n), float(T))


def hermite_E(i, j, t, Xab, a, b) -> float:
    """E^{ij}_t for one axis, Xab = A_x - B_x (Eqs. recurrence-A/B)."""
    return lib().orc_hermite_E(int(i), int(j), int(t), float(Xab), float(a), float(b))


def hermite_R(n, t, u, v, a, X, Y, Z) -> float:
    """R^n_tuv(a, (X, Y, Z)) (Eq. R-recursion)."""
    return lib().orc_hermite_R(int(n), int(t), int(u), int(v), float(a), float(X), float(Y), float(Z))


def jacobi_eigh(A: np.ndarray):
    """Eigenpairs of a symmetric matrix by cyclic Jacobi: (w ascending, V)."""
    n = A.shape[0]
    W = np.ascontiguousarray(A, dtype=np.float64).copy()
    w = np.zeros(n)
    V = np.zeros((n, n))
    lib().orc_jacobi_eigh(n, W, w, V)
    return w, V


class OracleBasis:
    """A normalised contracted Cartesian basis on the oracle side."""

    def __init__(self, mol):
        a = mol.arrays()
        self._keep = a
        self.mol = mol
        self.h = lib().orc_basis_create(mol.natom, a["Z"], a["xyz"].reshape(-1), mol.nshell,
                                        a["shell_atom"], a["shell_l"], a["shell_nprim"],
                                        a["alpha"], a["coef"])
        self.nbf = lib().orc_basis_nbf(self.h)
        self.shell_l = a["shell_l"]
        ao = np.zeros(mol.nshell, dtype=np.int64)
        off = 0
        for i, l in enumerate(self.shell_l):
            ao[i] = off
            off += (l + 1) * (l + 2) // 2
        self.ao = ao

    def __del__(self):
        try:
            if self.h:
                lib().orc_basis_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def onee(self, which: str) -> np.ndarray:
        code = {"S": 0, "T": 1, "V": 2}[which]
        out = np.zeros((self.nbf, self.nbf))
        lib().orc_onee(self.h, code, out)
        return out

    def enuc(self) -> float:
        return lib().orc_enuc(self.h)

    def eri_block(self, a, b, c, d) -> np.ndarray:
        n = [(int(self.shell_l[s]) + 1) * (int(self.shell_l[s]) + 2) // 2 for s in (a, b, c, d)]
        out = np.zeros(int(np.prod(n)))
        lib().orc_eri_shell_quartet(self.h, int(a), int(b), int(c), int(d), out)
        return out.reshape(n)

    def eri_blocks(self, quartets) -> list:
        """Blocks of a list of shell quartets (same layout as eri_block), OpenMP over the list."""
        q = np.ascontiguousarray(np.asarray(quartets, dtype=np.int32).reshape(-1, 4))
        nc = (np.asarray(self.shell_l)[q] + 1) * (np.asarray(self.shell_l)[q] + 2) // 2
        sizes = np.prod(nc, axis=1).astype(np.int64)
        off = np.ascontiguousarray(np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64))
        out = np.zeros(int(sizes.sum()))
        lib().orc_eri_quartet_list(self.h, len(q), q, off.ctypes.data_as(C.POINTER(C.c_longlong)), out)
        return [out[o:o + n].reshape(tuple(c)) for o, n, c in zip(off, sizes, nc)]

    def eri_full(self) -> np.ndarray:
        N = self.nbf
        g = np.zeros(N ** 4)
        lib().orc_eri_full(self.h, g)
        return g.reshape(N, N, N, N)

    def schwarz(self) -> np.ndarray:
        ns = self.mol.nshell
        Q = np.zeros(ns * ns)
        lib().orc_schwarz(self.h, Q)
        return Q.reshape(ns, ns)

    def jk_block(self, D: np.ndarray, sa: int, sb: int, tau: float = 0.0, Q=None):
        """(J_ab, K_ab) blocks for shells (sa, sb) by definition (all ordered kets)."""
        la, lb = int(self.shell_l[sa]), int(self.shell_l[sb])
        na, nb = (la + 1) * (la + 2) // 2, (lb + 1) * (lb + 2) // 2
        D = np.ascontiguousarray(D, dtype=np.float64)
        Jb = np.zeros(na * nb)
        Kb = np.zeros(na * nb)
        if Q is None:
            Q = np.zeros(1) if tau <= 0 else self.schwarz()
        Q = np.ascontiguousarray(Q, dtype=np.float64).reshape(-1)
        lib().orc_jk_block(self.h, D, int(sa), int(sb), Jb, Kb, float(tau), Q)
        return Jb.reshape(na, nb), Kb.reshape(na, nb)

    def jk_sample(self, D: np.ndarray, tau: float, bra_stride: int, nthreads: int = 0):
        """J/K contributions of the bra pairs ij with ij % bra_stride == 0 (timing sample)."""
        N = self.nbf
        D = np.ascontiguousarray(D, dtype=np.float64)
        J = np.zeros((N, N))
        K = np.zeros((N, N))
        nq = C.c_longlong(0)
        lib().orc_jk_sample(self.h, D, J, K, float(tau), int(nthreads), C.byref(nq), int(bra_stride))
        return J, K, nq.value

    def jk_shard(self, D: np.ndarray, shard: int, nshards: int, tau: float = 0.0, nthreads: int = 0):
        """J/K contributions of the bra pairs ij with ij % nshards == shard."""
        N = self.nbf
        D = np.ascontiguousarray(D, dtype=np.float64)
        J = np.zeros((N, N))
        K = np.zeros((N, N))
        nq = C.c_longlong(0)
        lib().orc_jk_shard(self.h, D, J, K, float(tau), int(nthreads), C.byref(nq), int(shard), int(nshards))
        return J, K, nq.value

    def jk(self, D: np.ndarray, tau: float = 0.0, nthreads: int = 0):
        """(J, K, n_unique_quartets_evaluated) over unique shell quartets."""
        N = self.nbf
        D = np.ascontiguousarray(D, dtype=np.float64)
        J = np.zeros((N, N))
        K = np.zeros((N, N))
        nq = C.c_longlong(0)
        lib().orc_jk(self.h, D, J, K, float(tau), int(nthreads), C.byref(nq))
        return J, K, nq.value
