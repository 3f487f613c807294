"""Pins of the FP64 oracle against what the mathematics fixes.

The paper (arxiv 2407.08092) prints no worked example, vectors, residuals or
eigenvalues, so every pin here is a closed form, an invariant or brute-force
dense linear algebra on a tiny lattice.  Each is chosen so that a plausible
mistake in the oracle -- a dropped term, a wrong sign or index, a transposed
operand, a wrong normalisation -- fails at least one of them.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import EVEN, ODD
from paper_2407_08092_gb300 import synth


def coords(L):
    x = np.arange(int(np.prod(L)))
    return np.stack([x % L[0], (x // L[0]) % L[1], (x // (L[0] * L[1])) % L[2],
                     x // (L[0] * L[1] * L[2])], axis=1)


def rand_lattice(L, seed=7, eps=0.5, m0=0.05, csw=1.0, t_bc=-1):
    return oracle.Lattice(L, synth.gauge_links(L, eps, seed), m0=m0, csw=csw, t_bc=t_bc)


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


# ---------------------------------------------------------------------------
# gamma matrices and links
# ---------------------------------------------------------------------------

def test_gamma_clifford_and_chiral():
    g = [oracle.gamma(m) for m in range(4)]
    for m, n in itertools.product(range(4), repeat=2):
        anti = g[m] @ g[n] + g[n] @ g[m]
        assert np.allclose(anti, 2.0 * (m == n) * np.eye(4), atol=1e-15)
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T, atol=1e-15)   # Hermitian
    g5 = oracle.gamma(4)
    assert np.allclose(g5, g[0] @ g[1] @ g[2] @ g[3], atol=1e-15)
    # chiral basis: gamma_5 = diag(1, 1, -1, -1), so the clover splits into 6x6 blocks
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=1e-15)


def test_links_are_su3_and_seeded():
    L = (4, 4, 2, 2)
    U = synth.gauge_links(L, 0.25, 123).reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.abs(np.einsum("nab,ncb->nac", U, U.conj()) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1.0).max() < 1e-14
    assert np.array_equal(U, synth.gauge_links(L, 0.25, 123).reshape(-1, 3, 3))
    assert not np.array_equal(U, synth.gauge_links(L, 0.25, 124).reshape(-1, 3, 3))
    # the generator is exp(i eps sum a_k lambda_k): for small eps, U ~ 1 + i eps H
    a = np.random.default_rng(3).standard_normal((5, 8))
    small = synth.su3_from_algebra(a, 1e-7)
    H = np.einsum("nk,kab->nab", a, synth.gell_mann())
    assert np.abs(small - (np.eye(3) + 1e-7j * H)).max() < 1e-13


# ---------------------------------------------------------------------------
# free field: plane waves and the Schur-complement spectrum
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("t_bc", [-1, +1])
def test_free_field_plane_wave(t_bc):
    """U = 1: psi(x) = e^{ip.x} u with p_k = 2 pi n_k / L_k and
    p_4 = (2n + (1 - t_bc)/2) pi / L_4 obeys
    D psi = [m0 + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu] psi.
    The clover term vanishes on the free field, so csw is irrelevant."""
    L = (4, 6, 2, 4)
    m0 = 0.137
    lat = oracle.Lattice(L, synth.unit_links(L), m0=m0, csw=1.3, t_bc=t_bc)
    c = coords(L)
    g = [oracle.gamma(m) for m in range(4)]
    rng = np.random.default_rng(11)
    shift = 0.5 * (1 - t_bc)
    for n in [(0, 0, 0, 0), (1, 2, 1, 3), (3, 5, 0, 1), (2, 1, 1, 2)]:
        p = np.array([2 * np.pi * n[0] / L[0], 2 * np.pi * n[1] / L[1],
                      2 * np.pi * n[2] / L[2], (2 * n[3] + shift) * np.pi / L[3]])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (c @ p))
        psi = phase[:, None, None] * u[None]
        M = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(g[m] * np.sin(p[m]) for m in range(4))
        expect = phase[:, None, None] * (M @ u)[None]
        assert np.abs(lat.dirac(psi) - expect).max() < 1e-13


def _free_schur_eigs(L, m0):
    """spec(D_S) on the free field: a - kappa^2/a, a = 4 + m0,
    kappa = sum cos p_mu +- i sqrt(sum sin^2 p_mu); every (p, +-) over the
    full antiperiodic-in-time zone carries multiplicity 3 (p and p + (pi,pi,pi,pi)
    share one even-site eigenspace of dimension 6)."""
    a = 4.0 + m0
    out = []
    for n in itertools.product(*(range(v) for v in L)):
        p = [2 * np.pi * n[k] / L[k] for k in range(3)] + [(2 * n[3] + 1) * np.pi / L[3]]
        cs = sum(np.cos(q) for q in p)
        sn = np.sqrt(sum(np.sin(q) ** 2 for q in p))
        for sgn in (+1, -1):
            kap = cs + sgn * 1j * sn
            out += [a - kap * kap / a] * 3
    return np.array(out)


def _match_multiset(a, b):
    """max distance after matching two complex multisets by sorting on a rounded key."""
    key = lambda z: np.lexsort((np.round(z.imag, 8), np.round(z.real, 8)))  # noqa: E731
    return np.abs(a[key(a)] - b[key(b)]).max()


@pytest.mark.parametrize("L", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_free_schur_spectrum(L):
    m0 = 0.05
    lat = oracle.Lattice(L, synth.unit_links(L), m0=m0, csw=1.0, t_bc=-1)
    DS = oracle.dense(lat.schur, 12 * lat.Vh, (lat.Vh, 4, 3))
    ev = np.linalg.eigvals(DS)
    expect = _free_schur_eigs(L, m0)
    assert len(ev) == len(expect)
    assert _match_multiset(ev, expect) < 1e-10


# ---------------------------------------------------------------------------
# structure on random gauge fields
# ---------------------------------------------------------------------------

def test_gamma5_hermiticity():
    """<phi, D psi> = <g5 D g5 phi, psi> for D and for D_S (random U, clover on)."""
    L = (4, 4, 2, 4)
    lat = rand_lattice(L, seed=21, eps=0.6, csw=1.7)
    rng = np.random.default_rng(5)
    for n, op in ((lat.V, lat.dirac), (lat.Vh, lat.schur)):
        phi = rng.standard_normal((n, 4, 3)) + 1j * rng.standard_normal((n, 4, 3))
        psi = rng.standard_normal((n, 4, 3)) + 1j * rng.standard_normal((n, 4, 3))
        lhs = np.vdot(phi, op(psi))
        rhs = np.vdot(lat.g5(op(lat.g5(phi))), psi)
        assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    # and densely on 2^4: D^+ = g5 D g5 exactly
    small = rand_lattice((2, 2, 2, 2), seed=22, eps=0.8, csw=1.2)
    D = oracle.dense(small.dirac, 12 * small.V, (small.V, 4, 3))
    G5 = np.kron(np.eye(small.V), np.kron(oracle.gamma(4), np.eye(3)))
    assert np.abs(D.conj().T - G5 @ D @ G5).max() < 1e-14


def test_gauge_covariance():
    """U'_mu(x) = W(x) U_mu(x) W(x+mu)^+  =>  D[U'] (W psi) = W (D[U] psi) and
    C'(x) = W C(x) W^+ (W acting on colour)."""
    L = (4, 2, 4, 4)
    U = synth.gauge_links(L, 0.7, 31)
    W = synth.random_gauge_transform(L, 32)
    c = coords(L)
    Up = np.empty_like(U)
    for mu in range(4):
        cn = c.copy()
        cn[:, mu] = (cn[:, mu] + 1) % L[mu]
        nb = cn[:, 0] + L[0] * (cn[:, 1] + L[1] * (cn[:, 2] + L[2] * cn[:, 3]))
        Up[:, mu] = np.einsum("nab,nbc,ndc->nad", W, U[:, mu], W[nb].conj())
    lat = oracle.Lattice(L, U, m0=-0.2, csw=1.4, t_bc=-1)
    latp = oracle.Lattice(L, Up, m0=-0.2, csw=1.4, t_bc=-1)
    rng = np.random.default_rng(6)
    psi = rng.standard_normal((lat.V, 4, 3)) + 1j * rng.standard_normal((lat.V, 4, 3))
    Wpsi = np.einsum("nab,nsb->nsa", W, psi)
    lhs = latp.dirac(Wpsi)
    rhs = np.einsum("nab,nsb->nsa", W, lat.dirac(psi))
    assert rel(lhs, rhs) < 1e-13
    Wbig = np.einsum("st,nab->nsatb", np.eye(4), W).reshape(lat.V, 12, 12)
    Crot = np.einsum("nij,njk,nlk->nil", Wbig, lat.C, Wbig.conj())
    assert np.abs(latp.C - Crot).max() < 1e-13


def test_clover_abelian_closed_form():
    """Constant abelian field strength in the (x,y) and (z,t) planes.

    Links: U_x(x) = exp(-i th Lam y), U_z(x) = exp(-i ph Lam' t), U_y = U_t = 1,
    with Lam = diag(1,-1,0), Lam' = diag(0,1,-1), th = 2 pi / L_y, ph = 4 pi / L_t
    (periodic links).  Every counter-clockwise leaf in the (x,y) plane is then
    exp(i th Lam), so Q_xy = 4 exp(i th Lam) and F_xy = (Q - Q^+)/8 = i sin(th Lam);
    likewise F_zt = i sin(ph Lam'); all other planes vanish.  With
    sigma_mu_nu = (i/2)[g_mu, g_nu] in the chiral basis,
    sigma_xy = diag(-1, 1, -1, 1) and sigma_zt = diag(1, -1, -1, 1) (spin), so
    C = (4 + m0) - (csw/2) [sigma_xy (x) sin(th Lam) + sigma_zt (x) sin(ph Lam')],
    a diagonal matrix independent of the site and of the fermion boundary."""
    L = (4, 6, 2, 4)
    m0, csw = 0.3, 1.25
    th, ph = 2 * np.pi / L[1], 4 * np.pi / L[3]
    Lam, Lamp = np.array([1.0, -1.0, 0.0]), np.array([0.0, 1.0, -1.0])
    c = coords(L)
    U = synth.unit_links(L)
    U[:, 0] = np.einsum("na,ab->nab", np.exp(-1j * th * np.outer(c[:, 1], Lam)), np.eye(3))
    U[:, 2] = np.einsum("na,ab->nab", np.exp(-1j * ph * np.outer(c[:, 3], Lamp)), np.eye(3))
    sxy = np.array([-1.0, 1.0, -1.0, 1.0])
    szt = np.array([1.0, -1.0, -1.0, 1.0])
    diag = (4 + m0) - 0.5 * csw * (np.outer(sxy, np.sin(th * Lam)) + np.outer(szt, np.sin(ph * Lamp)))
    expect = np.diag(diag.reshape(12))
    for t_bc in (-1, +1):
        lat = oracle.Lattice(L, U, m0=m0, csw=csw, t_bc=t_bc)
        assert np.abs(lat.C - expect[None]).max() < 1e-14
    # csw = 0 is the plain Wilson operator: C = (4 + m0) 1
    lat0 = oracle.Lattice(L, U, m0=m0, csw=0.0)
    assert np.abs(lat0.C - (4 + m0) * np.eye(12)[None]).max() < 1e-15


def test_clover_from_paired_leaves():
    """C(x) rebuilt from the field strength written with the leaves paired by a
    shared link (only F = (Q - Q^+)/8 is needed, so with AH(M) = M - M^+:
    F = [AH(U_mu(x) (A - B)) + AH((C' - D') U_mu(x - mu))] / 8, where
    L1 = U_mu(x) A, L4^+ = U_mu(x) B, L2 = C' U_mu(x - mu), L3^+ = D' U_mu(x - mu))
    and C = (4 + m0) + c_sw (i/2) sum_{mu<nu} sigma_mu_nu (x) F_mu_nu equals the
    oracle's clover term, which sums the four leaves directly."""
    L = (4, 4, 2, 6)
    lat = rand_lattice(L, seed=43, eps=0.7, csw=1.3)
    U, c = lat.U, coords(L)
    dag = lambda m: np.conj(np.swapaxes(m, -1, -2))

    def at(d, mu):   # U_mu at x + d for every site x
        cc = (c + np.asarray(d)) % np.asarray(L)
        return U[cc[:, 0] + L[0] * (cc[:, 1] + L[1] * (cc[:, 2] + L[2] * cc[:, 3])), mu]

    def e(mu, k=1):
        v = np.zeros(4, dtype=int)
        v[mu] = k
        return v

    mm = lambda *ms: ms[0] if len(ms) == 1 else np.einsum("nab,nbc->nac", ms[0], mm(*ms[1:]))
    g = [oracle.gamma(mu) for mu in range(4)]
    C = np.zeros((lat.V, 12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            m, n = e(mu), e(nu)
            A = mm(at(m, nu), dag(at(n, mu)), dag(at(0 * m, nu)))
            B = mm(dag(at(m - n, nu)), dag(at(-n, mu)), at(-n, nu))
            Cp = mm(at(0 * m, nu), dag(at(n - m, mu)), dag(at(-m, nu)))
            Dp = mm(dag(at(-n, nu)), dag(at(-m - n, mu)), at(-m - n, nu))
            M1 = mm(at(0 * m, mu), A - B)
            M2 = mm(Cp - Dp, at(-m, mu))
            F = (M1 - dag(M1) + M2 - dag(M2)) / 8
            sigma = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
            C += 0.5j * lat.csw * np.einsum("st,nab->nsatb", sigma, F).reshape(lat.V, 12, 12)
    C += (4 + lat.m0) * np.eye(12)
    assert np.abs(C - lat.C).max() < 1e-13
    assert np.abs(lat.C - (4 + lat.m0) * np.eye(12)).max() > 1e-2


def test_clover_from_rotated_plaquettes():
    """C(x) rebuilt from plaquettes only, in three passes: each leaf at x is the
    plaquette of a neighbouring corner rotated to start at x, and the
    anti-Hermitian part AH(M) = M - M^+ commutes with that unitary rotation, so
    with P(y) = U_mu(y) U_nu(y+mu) U_mu(y+nu)^+ U_nu(y)^+:
      R(y) = AH(P(y)) + U_mu(y-mu)^+ AH(P(y-mu)) U_mu(y-mu)      (leaves 1, 2)
      F(x) = [R(x) + U_nu(x-nu)^+ R(x-nu) U_nu(x-nu)] / 8        (leaves 1..4)
    and C = (4 + m0) + c_sw (i/2) sum_{mu<nu} sigma_mu_nu (x) F_mu_nu equals the
    oracle's clover term, which sums the four leaves directly."""
    L = (4, 2, 4, 6)
    lat = rand_lattice(L, seed=47, eps=0.7, csw=1.3)
    U, c = lat.U, coords(L)
    dag = lambda m: np.conj(np.swapaxes(m, -1, -2))
    mm = lambda *ms: ms[0] if len(ms) == 1 else np.einsum("nab,nbc->nac", ms[0], mm(*ms[1:]))
    AH = lambda m: m - dag(m)

    def idx(d):      # the site x + d of every site x
        cc = (c + np.asarray(d)) % np.asarray(L)
        return cc[:, 0] + L[0] * (cc[:, 1] + L[1] * (cc[:, 2] + L[2] * cc[:, 3]))

    def e(mu, k=1):
        v = np.zeros(4, dtype=int)
        v[mu] = k
        return v

    g = [oracle.gamma(mu) for mu in range(4)]
    C = np.zeros((lat.V, 12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            m, n = e(mu), e(nu)
            Umu, Unu = U[:, mu], U[:, nu]
            P = mm(Umu, Unu[idx(m)], dag(Umu[idx(n)]), dag(Unu))
            Hp = AH(P)
            W = Umu[idx(-m)]
            R = Hp + mm(dag(W), Hp[idx(-m)], W)
            W = Unu[idx(-n)]
            F = (R + mm(dag(W), R[idx(-n)], W)) / 8
            sigma = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
            C += 0.5j * lat.csw * np.einsum("st,nab->nsatb", sigma, F).reshape(lat.V, 12, 12)
    C += (4 + lat.m0) * np.eye(12)
    assert np.abs(C - lat.C).max() < 1e-13
    assert np.abs(lat.C - (4 + lat.m0) * np.eye(12)).max() > 1e-2


def test_clover_structure_and_inverse():
    """C is Hermitian, commutes with g5 (two 6x6 blocks), and C C^{-1} = 1."""
    lat = rand_lattice((4, 4, 4, 2), seed=41, eps=0.9, csw=1.9)
    C, Ci = lat.C, lat.Cinv
    assert np.abs(C - C.conj().transpose(0, 2, 1)).max() < 1e-14
    G5 = np.kron(oracle.gamma(4), np.eye(3))
    assert np.abs(G5 @ C - C @ G5).max() < 1e-14
    assert np.abs(C[:, :6, 6:]).max() < 1e-15 and np.abs(C[:, 6:, :6]).max() < 1e-15
    assert np.abs(np.einsum("nij,njk->nik", C, Ci) - np.eye(12)).max() < 1e-14
    # the field strength is not trivially zero on this field
    assert np.abs(C - (4 + lat.m0) * np.eye(12)).max() > 1e-2
    # sampled clover equals the full one
    sites = np.array([0, 5, 17, lat.V - 1])
    assert np.abs(lat.clover_sites(sites) - C[sites]).max() == 0.0


def test_inverse_against_library():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((20, 12, 12)) + 1j * rng.standard_normal((20, 12, 12))
    assert np.abs(oracle.invert(A) - np.linalg.inv(A)).max() < 1e-11


# ---------------------------------------------------------------------------
# odd-even reordering, Eq. 1-3
# ---------------------------------------------------------------------------

def test_odd_even_against_dense_lu():
    """On 2^4 (D is 192 x 192): the factorised inverse of Eq. 2 (prepare, dense
    D_S solve, reconstruct) gives the same x as a dense LU solve of D x = b, and
    the Schur complement assembled from the dense blocks of D (Eq. 1, Eq. 3)
    equals the matrix-free D_S."""
    lat = rand_lattice((2, 2, 2, 2), seed=51, eps=0.7, csw=1.3, m0=-0.1)
    D = oracle.dense(lat.dirac, 12 * lat.V, (lat.V, 4, 3))
    rng = np.random.default_rng(9)
    b = rng.standard_normal((lat.V, 4, 3)) + 1j * rng.standard_normal((lat.V, 4, 3))
    x_lu = np.linalg.solve(D, b.reshape(-1)).reshape(lat.V, 4, 3)
    assert rel(lat.dirac(x_lu), b) < 1e-13

    DS = oracle.dense(lat.schur, 12 * lat.Vh, (lat.Vh, 4, 3))
    xe = np.linalg.solve(DS, lat.prepare(b).reshape(-1)).reshape(lat.Vh, 4, 3)
    x_oe = lat.reconstruct(b, xe)
    assert rel(x_oe, x_lu) < 1e-13

    idx = [np.concatenate([np.arange(12 * s, 12 * s + 12) for s in lat.sites[p]]) for p in (EVEN, ODD)]
    Dee, Deo = D[np.ix_(idx[0], idx[0])], D[np.ix_(idx[0], idx[1])]
    Doe, Doo = D[np.ix_(idx[1], idx[0])], D[np.ix_(idx[1], idx[1])]
    assert np.abs(DS - (Dee - Deo @ np.linalg.solve(Doo, Doe))).max() < 1e-13
    # D_ee, D_oo block diagonal with 12x12 (two 6x6) blocks: no hopping inside a parity
    offdiag = Dee.copy()
    for s in range(lat.Vh):
        offdiag[12 * s:12 * s + 12, 12 * s:12 * s + 12] = 0
    assert np.abs(offdiag).max() == 0.0


def test_schur_sampled_sites_match_full():
    lat = rand_lattice((4, 4, 2, 4), seed=61, eps=0.5, csw=1.0)
    rng = np.random.default_rng(4)
    xe = rng.standard_normal((lat.Vh, 4, 3)) + 1j * rng.standard_normal((lat.Vh, 4, 3))
    full = lat.schur(xe)
    sel = np.array([0, 1, 7, 31, lat.Vh - 1])
    assert rel(lat.schur_sites(xe, sel), full[sel]) < 1e-14


# ---------------------------------------------------------------------------
# iterative methods, Algorithms 2 and 4, the smoother of Sec. 2.4.5
# ---------------------------------------------------------------------------

def _small_problem(seed=71):
    lat = rand_lattice((2, 2, 2, 2), seed=seed, eps=0.5, csw=1.0, m0=0.05)
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((lat.V, 4, 3)) + 1j * rng.standard_normal((lat.V, 4, 3))
    DS = oracle.dense(lat.schur, 12 * lat.Vh, (lat.Vh, 4, 3))
    return lat, b, DS


def test_richardson_polynomial_identity():
    """Sec. 2.4.5: after n sweeps from 0, x = p_{R,n}(D_S) b = (I - (I - w D_S)^n) D_S^{-1} b,
    i.e. the residual is (I - w D_S)^n b."""
    lat, b, DS = _small_problem()
    bh = lat.prepare(b).reshape(-1)
    omega = 0.8 / np.linalg.norm(DS, 2)
    for n in (1, 3, 5):
        x = lat_rich = oracle.richardson(lat.schur, bh.reshape(lat.Vh, 4, 3), omega, n)
        r_expect = np.linalg.matrix_power(np.eye(len(bh)) - omega * DS, n) @ bh
        assert rel(bh - DS @ lat_rich.reshape(-1), r_expect) < 1e-13
        p = (np.eye(len(bh)) - np.linalg.matrix_power(np.eye(len(bh)) - omega * DS, n)) @ np.linalg.inv(DS)
        assert rel(x.reshape(-1), p @ bh) < 1e-12


def test_gmres_one_cycle_is_krylov_minimiser():
    """One GMRES cycle of length m from x0 = 0 returns argmin ||b - A x|| over
    K_m(A, b) = span{b, Ab, ..., A^{m-1} b} (Sec. 2.4.2), here found by a dense
    QR least-squares solve on the explicit Krylov matrix."""
    lat, b, DS = _small_problem(72)
    bh = lat.prepare(b).reshape(-1)
    for m in (1, 4, 7):
        x, info = oracle.gmres(lat.schur, bh.reshape(lat.Vh, 4, 3), m, 1, 0.0)
        K = np.stack([np.linalg.matrix_power(DS, j) @ bh for j in range(m)], axis=1)
        Q, R = np.linalg.qr(DS @ K)
        c = np.linalg.solve(R, Q.conj().T @ bh)
        assert rel(x.reshape(-1), K @ c) < 1e-9
        assert info["iters"] == m


def test_gmres_full_dimension_is_exact():
    """dim D_S = 96 on 2^4: GMRES(96) without restart solves exactly."""
    lat, b, DS = _small_problem(73)
    bh = lat.prepare(b)
    x, info = oracle.gmres(lat.schur, bh, 96, 1, 1e-13)
    assert info["rel_resid"] < 1e-12
    assert rel(x.reshape(-1), np.linalg.solve(DS, bh.reshape(-1))) < 1e-11


def test_gmres_restarted_and_breakdown():
    lat, b, DS = _small_problem(74)
    bh = lat.prepare(b)
    x, info = oracle.gmres(lat.schur, bh, 8, 200, 1e-10)
    assert info["converged"] and info["rel_resid"] <= 1e-10
    assert info["cycles"] > 1
    # a right-hand side that is an eigenvector: lucky breakdown after one step
    w, vecs = np.linalg.eig(DS)
    v = vecs[:, 0].reshape(lat.Vh, 4, 3)
    xv, iv = oracle.gmres(lat.schur, v, 10, 1, 1e-12)
    assert iv["iters"] == 1 and rel(xv, v / w[0]) < 1e-12


def test_fgmres_with_exact_and_richardson_preconditioner():
    lat, b, DS = _small_problem(75)
    bh = lat.prepare(b)
    DSi = np.linalg.inv(DS)
    exact = lambda v: (DSi @ v.reshape(-1)).reshape(v.shape)  # noqa: E731
    x, info = oracle.fgmres(lat.schur, bh, exact, 10, 3, 1e-12)
    assert info["iters"] == 1 and info["rel_resid"] < 1e-12
    omega = 0.8 / oracle.power_norm(lat.schur, lat.schur_dag, bh, 50)
    rich = lambda v: oracle.richardson(lat.schur, v, omega, 5)  # noqa: E731
    x2, info2 = oracle.fgmres(lat.schur, bh, rich, 10, 100, 1e-10)
    assert info2["converged"] and rel(x2.reshape(-1), DSi @ bh.reshape(-1)) < 1e-8


def test_power_norm_converges_to_two_norm():
    lat, b, DS = _small_problem(76)
    v0 = np.random.default_rng(1).standard_normal((lat.Vh, 4, 3)) + 0j
    smax = np.linalg.svd(DS, compute_uv=False)[0]
    est = oracle.power_norm(lat.schur, lat.schur_dag, v0, 300)
    assert abs(est - smax) < 1e-6 * smax
    # every estimate is a lower bound of ||D_S||_2 and |lambda_max| <= ||D_S||_2
    for k in (1, 2, 5):
        assert oracle.power_norm(lat.schur, lat.schur_dag, v0, k) <= smax * (1 + 1e-14)
    assert np.abs(np.linalg.eigvals(DS)).max() <= smax * (1 + 1e-14)


def test_smoother_against_dense_factorisation():
    """M_n of Fig. 1: Eq. 2 with D_S^{-1} replaced by p_{R,n}(D_S), built from the
    dense blocks of D and compared with the matrix-free smoother."""
    lat, b, DS = _small_problem(77)
    D = oracle.dense(lat.dirac, 12 * lat.V, (lat.V, 4, 3))
    idx = [np.concatenate([np.arange(12 * s, 12 * s + 12) for s in lat.sites[p]]) for p in (EVEN, ODD)]
    perm = np.concatenate(idx)
    Dp = D[np.ix_(perm, perm)]
    n2 = 12 * lat.Vh
    Dee, Deo, Doe, Doo = Dp[:n2, :n2], Dp[:n2, n2:], Dp[n2:, :n2], Dp[n2:, n2:]
    Dooi = np.linalg.inv(Doo)
    S = Dee - Deo @ Dooi @ Doe
    omega = 0.8 / np.linalg.norm(S, 2)
    n = 3
    I2 = np.eye(n2)
    p = (I2 - np.linalg.matrix_power(I2 - omega * S, n)) @ np.linalg.inv(S)
    Z = np.zeros((n2, n2))
    left = np.block([[I2, Z], [-Dooi @ Doe, I2]])
    mid = np.block([[p, Z], [Z, Dooi]])
    right = np.block([[I2, -Deo @ Dooi], [Z, I2]])
    M = left @ mid @ right
    e = oracle.smoother(lat, b, "richardson", n, omega=omega)
    e_dense = np.empty(12 * lat.V, dtype=complex)
    e_dense[perm] = M @ b.reshape(-1)[perm]
    assert rel(e.reshape(-1), e_dense) < 1e-12
    # a GMRES smoother with a full-dimension cycle is D^{-1} itself
    eg = oracle.smoother(lat, b, "gmres", 1, m=96)
    assert rel(eg.reshape(-1), np.linalg.solve(D, b.reshape(-1))) < 1e-10


def test_solve_reaches_tolerance_and_matches_dense():
    lat = rand_lattice((4, 2, 2, 4), seed=81, eps=0.4, csw=1.0, m0=0.05)
    rng = np.random.default_rng(81)
    b = rng.standard_normal((lat.V, 4, 3)) + 1j * rng.standard_normal((lat.V, 4, 3))
    D = oracle.dense(lat.dirac, 12 * lat.V, (lat.V, 4, 3))
    x_ref = np.linalg.solve(D, b.reshape(-1))
    for kw in ({"solver": "gmres", "restart": 10},
               {"solver": "fgmres", "restart": 10, "precond": "gmres", "smooth_n": 2, "smooth_m": 4}):
        x, info = oracle.solve(lat, b, tol=1e-10, max_restarts=200, **kw)
        # the tolerance is on the full system: ||b - D x|| <= 1e-10 ||b|| (up to the
        # rounding of the two residual evaluations)
        assert info["converged"] and info["rel_resid_true"] <= 1e-10 * (1 + 1e-6)
        assert rel(x.reshape(-1), x_ref) < 1e-8


def test_full_residual_is_the_schur_residual_after_reconstruction():
    """For any x_e, reconstructing x_o = D_oo^{-1}(b_o - D_oe x_e) (Eq. 2) leaves
    no odd residual, and the even residual of D x = b is b_hat_e - D_S x_e: the
    identity that lets the Schur solve stop on the full system's residual."""
    lat = rand_lattice((4, 2, 4, 2), seed=83, eps=0.4, csw=1.0, m0=0.05)
    rng = np.random.default_rng(83)
    b = rng.standard_normal((lat.V, 4, 3)) + 1j * rng.standard_normal((lat.V, 4, 3))
    xe = rng.standard_normal((lat.Vh, 4, 3)) + 1j * rng.standard_normal((lat.Vh, 4, 3))
    x = lat.reconstruct(b, xe)
    r = (b - lat.dirac(x)).reshape(lat.V, 4, 3)
    D = oracle.dense(lat.dirac, 12 * lat.V, (lat.V, 4, 3))
    r_dense = (b.reshape(-1) - D @ x.reshape(-1)).reshape(lat.V, 4, 3)
    assert rel(r, r_dense) < 1e-13
    odd, even = lat.sites[oracle.ODD], lat.sites[oracle.EVEN]
    assert np.abs(r[odd]).max() < 1e-13 * np.abs(b).max()
    assert rel(r[even], lat.prepare(b) - lat.schur(xe)) < 1e-13


def test_fig1_odd_even_shrinks_and_clusters_spectrum():
    """Qualitative claims of Sec. 2.4.5 / Fig. 1 (the paper's field is unknown):
    max |lambda(D_S)| < max |lambda(D)|, and D M_3 (odd-even Richardson) is
    clustered nearer 1 than D p_{R,3}(D) (plain Richardson)."""
    lat = rand_lattice((4, 4, 2, 2), seed=91, eps=0.5, csw=1.0, m0=-0.3)
    D = oracle.dense(lat.dirac, 12 * lat.V, (lat.V, 4, 3))
    DS = oracle.dense(lat.schur, 12 * lat.Vh, (lat.Vh, 4, 3))
    eD, eS = np.linalg.eigvals(D), np.linalg.eigvals(DS)
    assert np.abs(eS).max() < np.abs(eD).max()
    n, delta = 3, 1.0
    I = np.eye(D.shape[0])
    wD = delta / np.abs(eD).max()
    pD = (I - np.linalg.matrix_power(I - wD * D, n)) @ np.linalg.inv(D)
    wS = delta / np.abs(eS).max()
    M3 = oracle.dense(lambda r: oracle.smoother(lat, r, "richardson", n, omega=wS),
                      12 * lat.V, (lat.V, 4, 3))
    spread_plain = np.abs(np.linalg.eigvals(D @ pD) - 1).mean()
    spread_oe = np.abs(np.linalg.eigvals(D @ M3) - 1).mean()
    assert spread_oe < spread_plain
