"""Pins of the CPU FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against mathematics the paper fixes: a brute-force
evaluation of Eq. (3) with a differently-built epsilon tensor, 3x3 determinants
(numpy.linalg.det), an inverse lattice Fourier transform, the symmetries of the
epsilon contraction, lattice translations, colour rotations, a plane-wave closed
form, the mode-triplet ordering of Eq. (4), and compensated summation. A dropped
term, a wrong sign, a wrong index or a transposed operand in the oracle fails at
least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def site_coords(L):
    """Coordinates (x0, x1, x2) of every site, ordered x = x0 + L*(x1 + L*x2)."""
    x2, x1, x0 = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    return np.stack([x0.ravel(), x1.ravel(), x2.ravel()], axis=1)


def numpy_phases(L, momenta):
    """exp(-i 2 pi n.x / L) in floating point, straight from the definition."""
    c = site_coords(L).astype(np.float64)
    n = np.asarray(momenta, np.float64).reshape(-1, 3)
    return np.exp(-2j * np.pi * (n @ c.T) / L)


def levi_civita():
    eps = np.zeros((3, 3, 3))
    for a, b, c in itertools.product(range(3), repeat=3):
        eps[a, b, c] = (a - b) * (b - c) * (c - a) / 2.0
    return eps


def random_case(L, n_ev, nd, momenta, spins, coeffs, seed, orthonormal=True):
    rng = np.random.Generator(np.random.PCG64(seed))
    if orthonormal:
        V = workloads.eigenvectors(rng, L, n_ev)
    else:
        V = workloads.complex_gaussian(rng, (n_ev, L ** 3, 3))
    phis = [workloads.coefficients(rng, n_ev, d) for d in nd]
    return V, phis, np.asarray(momenta), np.asarray(spins), np.asarray(coeffs, np.complex128)


def brute_force_eq3(L, V, phis, momenta, spins, coeffs):
    """Eq. (3) summed over all (a, b, c) and all (l1, l2, l3), with no reconstruction step."""
    eps = levi_civita()
    n_ev = V.shape[0]
    ph = numpy_phases(L, momenta)
    coeffs = np.asarray(coeffs)
    nd = [p.shape[1] for p in phis]
    B = np.zeros((len(ph), nd[0], nd[1], nd[2]), np.complex128)
    for s, (al, be, ga) in enumerate(spins):
        Q1 = phis[0][al * n_ev:(al + 1) * n_ev]
        Q2 = phis[1][be * n_ev:(be + 1) * n_ev]
        Q3 = phis[2][ga * n_ev:(ga + 1) * n_ev]
        blk = np.einsum("px,abc,ld,me,nf,lxa,mxb,nxc->pdef", ph, eps, Q1, Q2, Q3, V, V, V,
                        optimize=True)
        c = coeffs[:, s][:, None, None, None] if coeffs.ndim == 2 else coeffs[s]
        B += c * blk
    return B


def numpy_q(V, phi, alpha):
    """q[x][a][d] by one numpy matrix product (library routine)."""
    n_ev = V.shape[0]
    Q = phi[alpha * n_ev:(alpha + 1) * n_ev]
    return np.einsum("lxa,ld->xad", V, Q)


def site_dets(V, phis, spins, coeffs):
    """sum_s c_s det[q1_al(x)[:, d1], q2_be(x)[:, d2], q3_ga(x)[:, d3]] for every site and d."""
    X = V.shape[1]
    nd = [p.shape[1] for p in phis]
    out = np.zeros((X, nd[0], nd[1], nd[2]), np.complex128)
    for s, (al, be, ga) in enumerate(spins):
        q1, q2, q3 = numpy_q(V, phis[0], al), numpy_q(V, phis[1], be), numpy_q(V, phis[2], ga)
        M = np.empty((X, nd[0], nd[1], nd[2], 3, 3), np.complex128)
        M[..., :, 0] = np.broadcast_to(q1.transpose(0, 2, 1)[:, :, None, None, :],
                                       (X, nd[0], nd[1], nd[2], 3))
        M[..., :, 1] = np.broadcast_to(q2.transpose(0, 2, 1)[:, None, :, None, :],
                                       (X, nd[0], nd[1], nd[2], 3))
        M[..., :, 2] = np.broadcast_to(q3.transpose(0, 2, 1)[:, None, None, :, :],
                                       (X, nd[0], nd[1], nd[2], 3))
        out += coeffs[s] * np.linalg.det(M)
    return out


# ---------------------------------------------------------------- phases, Eq. (2)

def test_phase_table_matches_definition():
    for L in (1, 2, 3, 5, 24):
        mom = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (-1, 0, 0), (0, -1, 2), (3, -2, 7)]
        ph = oracle.phase_table(L, mom)
        assert np.abs(ph - numpy_phases(L, mom)).max() < 1e-12
        assert np.allclose(ph[0], 1.0)
        # periodicity of the integer momentum: n and n + L give the same phases
        shifted = oracle.phase_table(L, [(m[0] + L, m[1] - L, m[2] + 2 * L) for m in mom])
        assert np.abs(shifted - ph).max() < 1e-15


def test_reconstruct_matches_matmul():
    V, phis, *_ = random_case(3, 7, (5, 4, 3), [(0, 0, 0)], [(0, 0, 0)], [1.0], seed=11)
    for al in range(4):
        q = oracle.reconstruct(V, phis[0], al)
        ref = (V.reshape(7, -1).T @ phis[0][al * 7:(al + 1) * 7]).reshape(27, 3, 5)
        assert rel(q, ref) < 1e-14


# ---------------------------------------------------------------- I1 brute force

@pytest.mark.parametrize("L", [1, 2, 3])
def test_bruteforce_eq3(L):
    mom = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, -1, 1)]
    spins = [(0, 1, 0), (1, 0, 0), (2, 3, 2), (3, 3, 1)]
    coeffs = [0.5, -0.5 + 0.25j, 0.5, -0.3j]
    n_ev = min(5, 3 * L ** 3)
    V, phis, mom, spins, coeffs = random_case(L, n_ev, (3, 4, 2), mom, spins, coeffs, seed=100 + L)
    B = oracle.bblock(L, V, *phis, mom, spins, coeffs)
    ref = brute_force_eq3(L, V, phis, mom, spins, coeffs)
    assert rel(B, ref) < 1e-13


def test_bruteforce_momentum_dependent_coefficients():
    L = 2
    mom = [(0, 0, 0), (1, 0, 0), (1, 1, 1)]
    spins = [(0, 1, 0), (2, 3, 2)]
    rng = np.random.default_rng(5)
    coeffs = rng.standard_normal((3, 2)) + 1j * rng.standard_normal((3, 2))
    V, phis, mom, spins, _ = random_case(L, 6, (3, 3, 3), mom, spins, [1, 1], seed=7)
    B = oracle.bblock(L, V, *phis, mom, spins, coeffs)
    ref = brute_force_eq3(L, V, phis, mom, spins, coeffs)
    assert rel(B, ref) < 1e-13


# ---------------------------------------------------------------- I2 determinants

def test_single_site_is_a_determinant():
    L, n_ev = 1, 3
    spins = [(0, 1, 2), (3, 3, 0)]
    coeffs = np.array([1.0, -0.7 + 0.2j])
    V, phis, mom, spins, coeffs = random_case(L, n_ev, (4, 3, 5), [(0, 0, 0), (1, 2, 3)],
                                              spins, coeffs, seed=3, orthonormal=False)
    B = oracle.bblock(L, V, *phis, mom, spins, coeffs)
    ref = site_dets(V, phis, spins, coeffs)[0]
    # on one site every momentum phase is e^0 = 1
    for p in range(len(mom)):
        assert rel(B[p], ref) < 1e-13


@pytest.mark.parametrize("L", [2, 3])
def test_inverse_dft_recovers_site_determinants(L):
    """L^-3 sum_p e^{+i p.y} B^{(p)} = per-site determinant sum at site y (all L^3 momenta)."""
    mom = site_coords(L)  # every integer momentum mod L
    spins = [(0, 1, 0), (2, 2, 3)]
    coeffs = np.array([0.6, -0.8j])
    V, phis, mom, spins, coeffs = random_case(L, 4, (2, 3, 2), mom, spins, coeffs, seed=21 + L)
    B = oracle.bblock(L, V, *phis, mom, spins, coeffs)
    ph = numpy_phases(L, mom)                    # (n_mom, X), e^{-i p.x}
    per_site = np.einsum("px,pdef->xdef", np.conj(ph), B) / L ** 3
    ref = site_dets(V, phis, spins, coeffs)
    assert rel(per_site, ref) < 1e-12


@pytest.mark.parametrize("L", [3, 4])
def test_row_factored_phase_reproduces_eq1(L):
    """The reading behind the FP16 form's row-factored path: for integer momenta,
    e^{-i p.x} = w^{n0 x0} w^{n1 x1 + n2 x2} with w = e^{-2 pi i / L}. Summing the site
    singlets of each lattice row (x1, x2) against w^{n0 x0} once per distinct n0 (mod L),
    then the rows against w^{n1 x1 + n2 x2}, gives Eq. (1) for every momentum, including
    components beyond L and negative ones, and momenta that share their n0."""
    mom = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
           (1, 1, 0), (-1, -1, 0), (L + 1, 2, -3)]
    spins = [(0, 1, 0), (1, 0, 0), (2, 3, 2)]
    coeffs = [0.5, -0.5, 0.3 + 0.2j]
    V, phis, mom, spins, coeffs = random_case(L, 5, (3, 4, 2), mom, spins, coeffs, seed=41 + L)
    B = oracle.bblock(L, V, *phis, mom, spins, coeffs)
    S = site_dets(V, phis, spins, coeffs).reshape(L, L, L, 3, 4, 2)   # [x2][x1][x0][d1][d2][d3]
    w = np.exp(-2j * np.pi / L)
    k = np.arange(L)
    # per lattice row, one sum per distinct n0
    rows = {n0: np.einsum("k,abkdef->abdef", w ** ((n0 * k) % L), S)
            for n0 in sorted({int(m[0]) % L for m in mom})}
    assert len(rows) < len(mom)
    x1, x2 = k[None, :], k[:, None]
    got = np.stack([np.einsum("ab,abdef->def", w ** ((int(n1) * x1 + int(n2) * x2) % L),
                              rows[int(n0) % L]) for n0, n1, n2 in mom])
    assert rel(got, B) < 1e-12


# ---------------------------------------------------------------- I3 antisymmetry

def _case_c1_like(seed, nd=(4, 5, 3), L=2, n_ev=5):
    mom = [(0, 0, 0), (1, 0, 1)]
    V, phis, mom, _, _ = random_case(L, n_ev, nd, mom, [(0, 0, 0)], [1.0], seed=seed)
    return L, V, phis, mom


def test_antisymmetry_under_line_exchange():
    L, V, (p1, p2, p3), mom = _case_c1_like(31)
    spins = np.array([(0, 1, 2), (3, 1, 1)])
    coeffs = np.array([0.9, -0.4 + 0.1j])
    B = oracle.bblock(L, V, p1, p2, p3, mom, spins, coeffs)
    # 1 <-> 2: sign -1, spins (alpha, beta) exchanged, indices d1 <-> d2
    B12 = oracle.bblock(L, V, p2, p1, p3, mom, spins[:, [1, 0, 2]], coeffs)
    assert rel(-B12.transpose(0, 2, 1, 3), B) < 1e-13
    # 2 <-> 3
    B23 = oracle.bblock(L, V, p1, p3, p2, mom, spins[:, [0, 2, 1]], coeffs)
    assert rel(-B23.transpose(0, 1, 3, 2), B) < 1e-13
    # 1 <-> 3
    B13 = oracle.bblock(L, V, p3, p2, p1, mom, spins[:, [2, 1, 0]], coeffs)
    assert rel(-B13.transpose(0, 3, 2, 1), B) < 1e-13
    # cyclic (1,2,3) -> (2,3,1): sign +1
    Bc = oracle.bblock(L, V, p2, p3, p1, mom, spins[:, [1, 2, 0]], coeffs)
    assert rel(Bc.transpose(0, 3, 1, 2), B) < 1e-13


def test_equal_lines_give_zero_on_the_diagonal():
    L, V, (p1, p2, p3), mom = _case_c1_like(32, nd=(4, 4, 3))
    B = oracle.bblock(L, V, p1, p1, p3, mom, [(2, 2, 0)], [1.0])
    scale = np.abs(B).max()
    for d in range(4):
        assert np.abs(B[:, d, d, :]).max() < 1e-14 * scale
    # and the whole block is antisymmetric in (d1, d2)
    assert rel(-B.transpose(0, 2, 1, 3), B) < 1e-13


# ---------------------------------------------------------------- I4 translation

@pytest.mark.parametrize("shift", [(1, 0, 0), (0, 2, 1), (2, 1, 2)])
def test_translation_multiplies_by_phase(shift):
    L = 3
    mom = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (-1, 2, 1)]
    V, phis, mom, spins, coeffs = random_case(L, 6, (3, 2, 3), mom, [(0, 1, 0), (1, 0, 3)],
                                              [0.5, -0.5], seed=41)
    B = oracle.bblock(L, V, *phis, mom, spins, coeffs)
    # V'(x) = V(x - a) with periodic wrap
    Vg = V.reshape(V.shape[0], L, L, L, 3)        # [l][x2][x1][x0][a]
    a = np.asarray(shift)
    Vs = np.roll(Vg, shift=(a[2], a[1], a[0]), axis=(1, 2, 3)).reshape(V.shape)
    Bs = oracle.bblock(L, Vs, *phis, mom, spins, coeffs)
    fac = np.exp(-2j * np.pi * (np.asarray(mom) @ a) / L)
    assert rel(Bs, fac[:, None, None, None] * B) < 1e-13


# ---------------------------------------------------------------- I5 trilinearity

def test_trilinearity_in_each_slot_and_coefficients():
    L = 2
    mom = [(0, 0, 0), (1, 1, 0)]
    V, phis, mom, spins, coeffs = random_case(L, 5, (3, 3, 2), mom, [(0, 1, 0), (2, 3, 1)],
                                              [0.7, -0.2j], seed=51)
    rng = np.random.default_rng(52)
    lam, mu = 0.3 - 1.1j, -0.8 + 0.4j
    for slot in range(3):
        other = workloads.coefficients(rng, 5, phis[slot].shape[1])
        a = list(phis); b = list(phis); c = list(phis)
        b[slot] = other
        c[slot] = lam * phis[slot] + mu * other
        Ba = oracle.bblock(L, V, *a, mom, spins, coeffs)
        Bb = oracle.bblock(L, V, *b, mom, spins, coeffs)
        Bc = oracle.bblock(L, V, *c, mom, spins, coeffs)
        assert rel(Bc, lam * Ba + mu * Bb) < 1e-13
    # linear in the spin coefficients: the block of a sum is the sum of single-triple blocks
    parts = [oracle.bblock(L, V, *phis, mom, spins[s:s + 1], coeffs[s:s + 1]) for s in range(2)]
    assert rel(oracle.bblock(L, V, *phis, mom, spins, coeffs), parts[0] + parts[1]) < 1e-13


# ---------------------------------------------------------------- I6 colour rotations

def _random_unitary(rng, n=3):
    z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def test_colour_su3_invariance_and_u3_determinant():
    L = 2
    mom = [(0, 0, 0), (1, 0, 0)]
    V, phis, mom, spins, coeffs = random_case(L, 6, (3, 2, 3), mom, [(0, 1, 2)], [1.0], seed=61)
    B = oracle.bblock(L, V, *phis, mom, spins, coeffs)
    rng = np.random.default_rng(62)
    U = np.stack([_random_unitary(rng) for _ in range(L ** 3)])
    U = U / np.linalg.det(U)[:, None, None] ** (1.0 / 3.0)      # SU(3) per site
    VU = np.einsum("xab,lxb->lxa", U, V)
    assert rel(oracle.bblock(L, VU, *phis, mom, spins, coeffs), B) < 1e-13
    # a constant U(3) rotation multiplies the block by det U
    W = _random_unitary(rng)
    VW = np.einsum("ab,lxb->lxa", W, V)
    assert rel(oracle.bblock(L, VW, *phis, mom, spins, coeffs), np.linalg.det(W) * B) < 1e-13


# ---------------------------------------------------------------- I7 plane waves

def test_plane_wave_closed_form():
    """V_l(x) = u_l e^{i 2 pi k_l.x/L}/sqrt(X): B^{(p)}_{l1l2l3} = X^{-1/2} det[u] [k1+k2+k3 = n_p mod L]."""
    L, n_ev = 3, 4
    X = L ** 3
    rng = np.random.default_rng(71)
    u = rng.standard_normal((3, n_ev)) + 1j * rng.standard_normal((3, n_ev))
    k = np.array([(0, 0, 0), (1, 0, 0), (2, 1, 0), (0, 2, 2)])
    c = site_coords(L)
    V = np.einsum("al,lx->lxa", u, np.exp(2j * np.pi * (k @ c.T) / L)) / math.sqrt(X)
    mom = [(0, 0, 0), (1, 0, 0), (3, 1, 0), (0, 0, 2), (2, 2, 2), (1, 1, 0)]
    eye = np.eye(n_ev)
    phi = np.zeros((4 * n_ev, n_ev), np.complex128)
    phi[0:n_ev] = eye                                  # spin 0 selects eigenvector d
    B = oracle.bblock(L, V, phi, phi, phi, mom, [(0, 0, 0)], [1.0])
    ref = np.zeros_like(B)
    for p, n in enumerate(mom):
        for l1, l2, l3 in itertools.product(range(n_ev), repeat=3):
            if np.all((k[l1] + k[l2] + k[l3] - np.asarray(n)) % L == 0):
                ref[p, l1, l2, l3] = np.linalg.det(u[:, [l1, l2, l3]]) / math.sqrt(X)
    assert np.abs(B - ref).max() < 1e-13 * max(1.0, np.abs(ref).max())
    assert np.abs(ref).max() > 0.1                     # the closed form is not trivially zero


# ---------------------------------------------------------------- I8 identity projection

def test_identity_projection_isolates_the_contraction():
    L = 2
    X = L ** 3
    n_ev = 3 * X
    V = np.eye(n_ev, dtype=np.complex128).reshape(n_ev, X, 3)
    rng = np.random.default_rng(81)
    phis = [workloads.coefficients(rng, n_ev, d) for d in (2, 3, 2)]
    for al in range(4):
        q = oracle.reconstruct(V, phis[1], al)
        assert np.array_equal(q, phis[1][al * n_ev:(al + 1) * n_ev].reshape(X, 3, 3))
    spins = [(1, 2, 3)]
    mom = [(0, 0, 0), (1, 0, 1)]
    B = oracle.bblock(L, V, *phis, mom, spins, [1.0])
    dets = site_dets(V, phis, spins, np.array([1.0]))
    ref = np.einsum("px,xdef->pdef", numpy_phases(L, mom), dets)
    assert rel(B, ref) < 1e-13


# ---------------------------------------------------------------- I9 mode-triplet ordering

def test_mode_triplet_is_totally_antisymmetric():
    L = 2
    V, _, mom, _, _ = random_case(L, 5, (1, 1, 1), [(0, 0, 0), (1, 0, 0)], [(0, 0, 0)], [1.0], 91)
    T = oracle.mode_triplet(L, V, mom)
    for perm, sign in (((0, 2, 1, 3), -1), ((0, 1, 3, 2), -1), ((0, 3, 2, 1), -1),
                       ((0, 2, 3, 1), 1), ((0, 3, 1, 2), 1)):
        assert rel(sign * T.transpose(perm), T) < 1e-14
    # only C(n_ev, 3) independent entries: repeated eigenvector indices vanish
    for l in range(5):
        assert np.abs(T[:, l, l, :]).max() < 1e-15


def test_direct_and_mode_triplet_orderings_agree_l4():
    w = workloads.WORKLOADS["l4_nev8_ndil8"]
    inp = workloads.generate(w)
    phis = [inp.phi[0][i][0] for i in range(3)]
    B = oracle.bblock(w.L, inp.V[0], *phis, inp.momenta, inp.spins, inp.coeffs)
    T = oracle.mode_triplet(w.L, inp.V[0], inp.momenta)
    B2 = oracle.bblock_via_triplet(T, *phis, inp.spins, inp.coeffs)
    assert rel(B, B2) < 1e-13


def test_direct_and_mode_triplet_orderings_agree_mixed_spins():
    L = 3
    mom = [(0, 0, 0), (1, 0, 0), (1, 1, 0)]
    spins = [(0, 1, 0), (1, 0, 0), (2, 3, 2)]
    coeffs = np.array([1, -1, 1]) / math.sqrt(2)
    V, phis, mom, spins, coeffs = random_case(L, 6, (4, 3, 5), mom, spins, coeffs, seed=92)
    B = oracle.bblock(L, V, *phis, mom, spins, coeffs)
    T = oracle.mode_triplet(L, V, mom)
    assert rel(oracle.bblock_via_triplet(T, *phis, spins, coeffs), B) < 1e-13


# ---------------------------------------------------------------- I11 oracle rounding

def test_compensated_summation_agrees():
    w = workloads.WORKLOADS["l4_nev8_ndil8"]
    inp = workloads.generate(w)
    phis = [inp.phi[0][i][0] for i in range(3)]
    qs = [oracle.reconstruct_all(inp.V[0], p) for p in phis]
    B = oracle.contract(w.L, *qs, inp.momenta, inp.spins, inp.coeffs)
    Bc = oracle.contract_compensated(w.L, *qs, inp.momenta, inp.spins, inp.coeffs)
    assert rel(B, Bc) < 1e-14


def test_compensated_summation_agrees_at_l24_sample():
    """At L=24 (13824 sites) the plain FP64 site sum stays within 1e-13 of a compensated one."""
    w = workloads.WORKLOADS["l24_nev96_ndil32"]
    inp = workloads.generate(w, n_t=1)
    cols = [[0, 17], [3, 31], [5, 9]]
    phis = [np.ascontiguousarray(inp.phi[0][i][0][:, cols[i]]) for i in range(3)]
    qs = [oracle.reconstruct_all(inp.V[0], p) for p in phis]
    B = oracle.contract(w.L, *qs, inp.momenta, inp.spins, inp.coeffs)
    Bc = oracle.contract_compensated(w.L, *qs, inp.momenta, inp.spins, inp.coeffs)
    assert rel(B, Bc) < 1e-13


def test_sampled_columns_equal_full_block():
    L = 2
    V, phis, mom, spins, coeffs = random_case(L, 5, (5, 4, 6), [(0, 0, 0), (0, 1, 1)],
                                              [(0, 1, 0), (1, 0, 2)], [0.5, -0.5], seed=95)
    B = oracle.bblock(L, V, *phis, mom, spins, coeffs)
    d1s, d2s, d3s = [4, 0], [1, 3], [5, 2, 0]
    S = oracle.bblock_sampled(L, V, *phis, mom, spins, coeffs, d1s, d2s, d3s)
    assert np.array_equal(S, B[:, d1s][:, :, d2s][:, :, :, d3s])


# ---------------------------------------------------------------- paper's printed sizes

def test_paper_object_sizes():
    g = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))
    d = g["diq"]
    values = d["BsizeD1"] * d["BsizeD2"] * d["n_colors"] * d["BsizeX"]
    assert values == d["values"]
    assert values * 16 == d["bytes_kB"] * 1024
    s = g["singlet"]
    assert s["BsizeD1"] * s["BsizeD2"] * s["BsizeD3"] * s["BsizeX"] * 16 == s["bytes_kB"] * 1024
    t = g["mode_triplet"]
    # the oracle's mode triplet is one n_ev^3 complex128 array per momentum
    V, _, mom, _, _ = random_case(1, 3, (1, 1, 1), [(0, 0, 0), (1, 0, 0)], [(0, 0, 0)], [1.0], 99)
    T = oracle.mode_triplet(1, V, mom)
    assert T.shape == (2, 3, 3, 3) and T.dtype == np.complex128
    tb = t["n_ev"] ** 3 * t["n_mom"] * T.itemsize / 2 ** 40
    assert abs(tb - t["TB"]) < 0.1
