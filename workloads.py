"""Seeded synthetic inputs for stochastic-LapH baryon blocks.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no reconstruction, no colour contraction, no phases). It is
the one piece that both the CPU oracle's tests and the CUDA path's tests and
benchmark use, so that both sides see identical bytes.

Recipe (real Laplacian eigenvectors, Dirac solves and group-theory spin
coefficients are not available, so these stand in for them):

* random stream: ``numpy.random.Generator(PCG64(seed))``; draws happen in a
  fixed order: for each time slice, V, then phi1, phi2, phi3 for each noise
  triple; the per-noise dilution sizes (batched workload) are drawn first;
* complex Gaussian entries: real and imaginary parts ~ N(0, 1/2) each;
* eigenvectors: a complex Gaussian (3 L^3) x N_ev matrix orthonormalised by
  Householder QR (``numpy.linalg.qr``), stored as ``V[l][x][a]`` with site
  ``x = x0 + L*(x1 + L*x2)`` and colour ``a``;
* quark-line coefficients ``phi[alpha*N_ev + l][d]``: (4 N_ev) x N_dil complex
  Gaussian (spin-major rows);
* momenta are integer triples ``n`` (``p = 2 pi n / L``) with ``|n|^2 <= 2``;
* spin operators are synthetic sets of spin triples with real coefficients.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 2211_16278

MOM_C2 = [(0, 0, 0), (1, 0, 0), (1, 1, 0)]
MOM_C3 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0)]
MOM_C5 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
MOM_C4 = MOM_C5 + [(1, 1, 0), (-1, -1, 0)]

_R2 = 1.0 / math.sqrt(2.0)
SPIN_C1 = ([(0, 0, 0)], [1.0])
SPIN_C2 = ([(0, 1, 0), (1, 0, 0), (2, 3, 2)], [_R2, -_R2, _R2])
SPIN_C3 = ([(0, 1, 0), (1, 0, 0), (2, 3, 2), (3, 2, 2)], [0.5, -0.5, 0.5, -0.5])


@dataclasses.dataclass(frozen=True)
class Workload:
    """Shape of one synthetic baryon-block run."""
    name: str
    L: int
    n_ev: int
    ndil: int                 # dilution size (per line) unless ``ndil_choices`` is set
    n_t: int
    momenta: Tuple[Tuple[int, int, int], ...]
    spins: Tuple[Tuple[int, int, int], ...]
    coeffs: Tuple[float, ...]
    n_noise: int = 1
    ndil_choices: Optional[Tuple[int, ...]] = None
    seed_index: int = 0

    @property
    def X(self) -> int:
        return self.L ** 3

    @property
    def seed(self) -> int:
        return SEED_BASE + self.seed_index

    def describe(self) -> str:
        nd = self.ndil_choices if self.ndil_choices else self.ndil
        return (f"L={self.L} (X={self.X}) N_ev={self.n_ev} N_dil={nd} n_t={self.n_t} "
                f"n_noise={self.n_noise} n_mom={len(self.momenta)} n_spin={len(self.spins)}")


def _w(name, L, n_ev, ndil, n_t, mom, spin, idx, **kw):
    return Workload(name, L, n_ev, ndil, n_t, tuple(map(tuple, mom)), tuple(map(tuple, spin[0])),
                    tuple(spin[1]), seed_index=idx, **kw)


WORKLOADS = {
    # one time slice, L=4, N_ev=8, N_dil=8, p=0, one spin triple
    "l4_nev8_ndil8": _w("l4_nev8_ndil8", 4, 8, 8, 1, [(0, 0, 0)], SPIN_C1, 1),
    # L=24, N_ev=96, N_dil=32, 8 time slices, 3 momenta, 3 spin triples
    "l24_nev96_ndil32": _w("l24_nev96_ndil32", 24, 96, 32, 8, MOM_C2, SPIN_C2, 2),
    # L=32, N_ev=128, N_dil=64, 16 time slices, 5 momenta, 4 spin triples
    "l32_nev128_ndil64": _w("l32_nev128_ndil64", 32, 128, 64, 16, MOM_C3, SPIN_C3, 3),
    # L=32, N_ev=128, 48 time slices x 9 momenta x 6 noise triples, N_dil in {32,48,64}
    "l32_batch_48t_6noise": _w("l32_batch_48t_6noise", 32, 128, 64, 48, MOM_C4, SPIN_C3, 4,
                               n_noise=6, ndil_choices=(32, 48, 64)),
    # L=48, N_ev=264, N_dil=64, 4 time slices, 7 momenta, 4 spin triples
    "l48_nev264_ndil64": _w("l48_nev264_ndil64", 48, 264, 64, 4, MOM_C5, SPIN_C3, 5),
}


def complex_gaussian(rng: np.random.Generator, shape) -> np.ndarray:
    """Entries with Re, Im ~ N(0, 1/2) independently."""
    s = math.sqrt(0.5)
    re = rng.standard_normal(shape) * s
    im = rng.standard_normal(shape) * s
    return re + 1j * im


def eigenvectors(rng: np.random.Generator, L: int, n_ev: int) -> np.ndarray:
    """Orthonormal complex vectors of length 3 L^3, returned as V[l][x][a]."""
    X = L ** 3
    if n_ev > 3 * X:
        raise ValueError("n_ev cannot exceed 3 L^3")
    g = complex_gaussian(rng, (3 * X, n_ev))
    q, _ = np.linalg.qr(g, mode="reduced")
    return np.ascontiguousarray(q.T.reshape(n_ev, X, 3))


def coefficients(rng: np.random.Generator, n_ev: int, ndil: int) -> np.ndarray:
    """phi[alpha*n_ev + l][d], shape (4 n_ev, ndil)."""
    return np.ascontiguousarray(complex_gaussian(rng, (4 * n_ev, ndil)))


@dataclasses.dataclass
class Inputs:
    """Host arrays of one run: V[t], phi[noise][line][t], per-noise dilution sizes."""
    workload: Workload
    V: np.ndarray                      # (n_t, n_ev, X, 3) complex128
    phi: List[List[np.ndarray]]        # [noise][line] -> (n_t, 4 n_ev, ndil) complex128
    ndil: List[Tuple[int, int, int]]   # (nd1, nd2, nd3) per noise triple
    momenta: np.ndarray                # (n_mom, 3) int32
    spins: np.ndarray                  # (n_spin, 3) int32
    coeffs: np.ndarray                 # (n_spin,) complex128


def generate(w: Workload, n_t: Optional[int] = None, seed: Optional[int] = None) -> Inputs:
    """Draw the inputs of workload ``w`` (optionally only its first ``n_t`` time slices).

    The draw order is fixed, so the first time slices are the same whether or not
    ``n_t`` truncates the run.
    """
    rng = np.random.Generator(np.random.PCG64(w.seed if seed is None else seed))
    nt_full = w.n_t
    nt = nt_full if n_t is None else min(n_t, nt_full)
    if w.ndil_choices:
        nds = [int(v) for v in rng.choice(np.asarray(w.ndil_choices), size=w.n_noise)]
    else:
        nds = [w.ndil] * w.n_noise
    V = np.empty((nt, w.n_ev, w.X, 3), np.complex128)
    phi = [[np.empty((nt, 4 * w.n_ev, nds[k]), np.complex128) for _ in range(3)]
           for k in range(w.n_noise)]
    for t in range(nt):
        V[t] = eigenvectors(rng, w.L, w.n_ev)
        for k in range(w.n_noise):
            for i in range(3):
                phi[k][i][t] = coefficients(rng, w.n_ev, nds[k])
    return Inputs(w, V, phi, [(n, n, n) for n in nds],
                  np.asarray(w.momenta, np.int32).reshape(-1, 3),
                  np.asarray(w.spins, np.int32).reshape(-1, 3),
                  np.asarray(w.coeffs, np.complex128))


def custom(L: int, n_ev: int, ndil: Sequence[int], n_t: int, momenta, spins, coeffs,
           seed: int) -> Inputs:
    """Inputs of an ad-hoc shape (tests): one noise triple with per-line ``ndil``."""
    nd = list(ndil) if hasattr(ndil, "__len__") else [ndil] * 3
    w = Workload(f"custom_L{L}", L, n_ev, nd[0], n_t, tuple(map(tuple, momenta)),
                 tuple(map(tuple, spins)), tuple(complex(c) for c in np.ravel(coeffs)))
    rng = np.random.Generator(np.random.PCG64(seed))
    V = np.empty((n_t, n_ev, L ** 3, 3), np.complex128)
    phi = [[np.empty((n_t, 4 * n_ev, nd[i]), np.complex128) for i in range(3)]]
    for t in range(n_t):
        V[t] = eigenvectors(rng, L, n_ev)
        for i in range(3):
            phi[0][i][t] = coefficients(rng, n_ev, nd[i])
    return Inputs(w, V, phi, [tuple(nd)], np.asarray(momenta, np.int32).reshape(-1, 3),
                  np.asarray(spins, np.int32).reshape(-1, 3), np.asarray(coeffs, np.complex128))
