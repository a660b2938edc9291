"""CPU FP64 oracle for stochastic-LapH baryon blocks (arXiv:2211.16278).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library never
imports, links or calls it, and it never calls the CUDA library: the two share
no code, header, table or helper.

The arithmetic lives in ``bblock_oracle.c`` (plain C99, ``double complex``, FP64,
OpenMP over the outer dilution loop). This module compiles it with gcc and wraps
each routine with ctypes, taking and returning numpy ``complex128`` arrays:

* :func:`phase_table`  -- e^{-i p.x}, p = 2 pi n / L, Eq. (1)/(3).
* :func:`reconstruct`  -- Eq. (2), one spin of one quark line.
* :func:`contract`     -- Eq. (1) given the reconstructed fields.
* :func:`bblock`       -- Eq. (2) then Eq. (1) for one time slice.
* :func:`mode_triplet` -- Eq. (4).
* :func:`bblock_via_triplet` -- Eq. (3) as T contracted with the coefficients.
* :func:`contract_compensated` -- Eq. (1) with compensated summation.

Layouts: ``V[l][x][a]`` (``n_ev, X, 3``), ``phi[alpha*n_ev + l][d]``
(``4*n_ev, ndil``), ``q[alpha][x][a][d]`` (``4, X, 3, ndil``),
``B[p][d1][d2][d3]``. Sites are ``x = x0 + L*(x1 + L*x2)``.

Parity status: every routine here is pinned by the CPU tests in
``tests/test_oracle_pins.py`` (brute force, determinants, symmetries, closed
forms); nothing in this file is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bblock_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lib = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the C oracle (gcc, -O3, OpenMP) into ``out``; default ``oracle/_build/liboracle.so``.

    No ``-march=native``: the same source must build and give the same results on the
    x86-64 development host and the Arm (Grace) GPU host."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-std=c99", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def load_library(path: str):
    """Open a compiled oracle library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i = ctypes.c_int
    l = ctypes.c_long
    lib.oracle_num_threads.restype = i
    lib.oracle_set_num_threads.argtypes = [i]
    lib.oracle_phase_table.argtypes = [i, i, P, P]
    lib.oracle_reconstruct.argtypes = [l, i, P, P, i, i, P]
    sig = [i, P, i, P, i, P, i, i, P, i, P, P, i, P]
    lib.oracle_contract.argtypes = sig
    lib.oracle_contract_compensated.argtypes = sig
    lib.oracle_bblock.argtypes = [i, i, P, P, i, P, i, P, i, i, P, i, P, P, i, P]
    lib.oracle_bblock.restype = i
    lib.oracle_mode_triplet.argtypes = [i, i, P, i, P, P]
    lib.oracle_bblock_via_triplet.argtypes = [i, P, P, i, P, i, P, i, i, i, P, P, i, P]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on (a timing control only)."""
    _load().oracle_set_num_threads(int(n))


def _spin_args(spin, coef, n_mom):
    spin = _c(np.asarray(spin).reshape(-1, 3), np.int32)
    coef = np.asarray(coef, dtype=np.complex128)
    per_mom = 1 if coef.ndim == 2 else 0
    if per_mom:
        assert coef.shape == (n_mom, spin.shape[0])
    else:
        assert coef.shape == (spin.shape[0],)
    return spin, _c(coef, np.complex128), per_mom


def phase_table(L: int, momenta) -> np.ndarray:
    mom = _c(np.asarray(momenta).reshape(-1, 3), np.int32)
    out = np.empty((mom.shape[0], L ** 3), np.complex128)
    _load().oracle_phase_table(L, mom.shape[0], _ptr(mom), _ptr(out))
    return out


def reconstruct(V, phi, alpha: int) -> np.ndarray:
    """Eq. (2): q[x][a][d] for spin ``alpha``. V is (n_ev, X, 3), phi (4*n_ev, ndil)."""
    V = _c(V, np.complex128)
    phi = _c(phi, np.complex128)
    n_ev, X, _ = V.shape
    ndil = phi.shape[1]
    assert phi.shape[0] == 4 * n_ev
    q = np.empty((X, 3, ndil), np.complex128)
    _load().oracle_reconstruct(X, n_ev, _ptr(V), _ptr(phi), ndil, alpha, _ptr(q))
    return q


def reconstruct_all(V, phi, spins=range(4)) -> np.ndarray:
    """q[alpha][x][a][d] for every alpha in ``spins`` (others left zero)."""
    V = np.asarray(V)
    q = np.zeros((4, V.shape[1], 3, np.asarray(phi).shape[1]), np.complex128)
    for al in sorted(set(int(s) for s in spins)):
        q[al] = reconstruct(V, phi, al)
    return q


def _contract(fn, L, q1, q2, q3, momenta, spin, coef):
    q1, q2, q3 = (_c(q, np.complex128) for q in (q1, q2, q3))
    mom = _c(np.asarray(momenta).reshape(-1, 3), np.int32)
    spin, coef, per_mom = _spin_args(spin, coef, mom.shape[0])
    nd = [q.shape[3] for q in (q1, q2, q3)]
    for q in (q1, q2, q3):
        assert q.shape[:3] == (4, L ** 3, 3)
    B = np.empty((mom.shape[0], nd[0], nd[1], nd[2]), np.complex128)
    fn(L, _ptr(q1), nd[0], _ptr(q2), nd[1], _ptr(q3), nd[2], mom.shape[0], _ptr(mom),
       spin.shape[0], _ptr(spin), _ptr(coef), per_mom, _ptr(B))
    return B


def contract(L, q1, q2, q3, momenta, spin, coef) -> np.ndarray:
    """Eq. (1) given q_i[alpha][x][a][d]. Returns B[p][d1][d2][d3]."""
    return _contract(_load().oracle_contract, L, q1, q2, q3, momenta, spin, coef)


def contract_compensated(L, q1, q2, q3, momenta, spin, coef) -> np.ndarray:
    """Eq. (1) with compensated summation (bounds the oracle's own rounding)."""
    return _contract(_load().oracle_contract_compensated, L, q1, q2, q3, momenta, spin, coef)


def bblock(L, V, phi1, phi2, phi3, momenta, spin, coef) -> np.ndarray:
    """Eq. (2) then Eq. (1) for one time slice. Returns B[p][d1][d2][d3]."""
    V = _c(V, np.complex128)
    phis = [_c(p, np.complex128) for p in (phi1, phi2, phi3)]
    n_ev = V.shape[0]
    assert V.shape == (n_ev, L ** 3, 3)
    for p in phis:
        assert p.shape[0] == 4 * n_ev
    mom = _c(np.asarray(momenta).reshape(-1, 3), np.int32)
    spin, coef, per_mom = _spin_args(spin, coef, mom.shape[0])
    nd = [p.shape[1] for p in phis]
    B = np.empty((mom.shape[0], nd[0], nd[1], nd[2]), np.complex128)
    rc = _load().oracle_bblock(L, n_ev, _ptr(V), _ptr(phis[0]), nd[0], _ptr(phis[1]), nd[1],
                               _ptr(phis[2]), nd[2], mom.shape[0], _ptr(mom), spin.shape[0],
                               _ptr(spin), _ptr(coef), per_mom, _ptr(B))
    if rc != 0:
        raise MemoryError("oracle_bblock: out of host memory")
    return B


def mode_triplet(L, V, momenta) -> np.ndarray:
    """Eq. (4): T[p][l1][l2][l3]."""
    V = _c(V, np.complex128)
    n_ev = V.shape[0]
    mom = _c(np.asarray(momenta).reshape(-1, 3), np.int32)
    T = np.empty((mom.shape[0], n_ev, n_ev, n_ev), np.complex128)
    _load().oracle_mode_triplet(L, n_ev, _ptr(V), mom.shape[0], _ptr(mom), _ptr(T))
    return T


def bblock_via_triplet(T, phi1, phi2, phi3, spin, coef) -> np.ndarray:
    """Eq. (3) as sum_s c_s T x1 phi1 x2 phi2 x3 phi3."""
    T = _c(T, np.complex128)
    n_mom, n_ev = T.shape[0], T.shape[1]
    phis = [_c(p, np.complex128) for p in (phi1, phi2, phi3)]
    spin, coef, per_mom = _spin_args(spin, coef, n_mom)
    nd = [p.shape[1] for p in phis]
    B = np.empty((n_mom, nd[0], nd[1], nd[2]), np.complex128)
    _load().oracle_bblock_via_triplet(n_ev, _ptr(T), _ptr(phis[0]), nd[0], _ptr(phis[1]), nd[1],
                                      _ptr(phis[2]), nd[2], n_mom, spin.shape[0], _ptr(spin),
                                      _ptr(coef), per_mom, _ptr(B))
    return B


def bblock_sampled(L, V, phi1, phi2, phi3, momenta, spin, coef, d1s, d2s, d3s) -> np.ndarray:
    """B[p][i][j][k] = B[p][d1s[i]][d2s[j]][d3s[k]] of one time slice.

    Selecting dilution columns commutes with Eq. (2) and Eq. (1) (both act on
    each column independently), so this evaluates the full definition on the
    column subsets; it is how full-size blocks are checked entry by entry.
    """
    sub = [np.ascontiguousarray(np.asarray(p)[:, list(ds)]) for p, ds in
           ((phi1, d1s), (phi2, d2s), (phi3, d3s))]
    return bblock(L, V, sub[0], sub[1], sub[2], momenta, spin, coef)
