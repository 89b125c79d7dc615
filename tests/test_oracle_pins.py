"""Pins of the CPU oracle against things other than itself (CPU only).

Each test names what fixes the expected value: a closed form, an identity of the mathematics,
brute-force quadrature written independently in ``tests/quadrature.py``, a library routine, or an
invariant of the method (Theory, "Fragment Mean Field").  The paper prints no numbers, so there is
no printed-value pin.
"""
import math

import numpy as np
import pytest

from oracle import integrals as I
from oracle.fef import Fragments, orthonormal_density, canonical_orthogonaliser
from synth import systems as S
from tests import quadrature as Q

BOHR = S.ANGSTROM_PER_BOHR


# ----------------------------------------------------------------------------------------- Boys

def test_boys_at_zero():
    """F_m(0) = 1/(2m+1)."""
    F = I.boys(16, 0.0)
    assert np.allclose(F, 1.0 / (2 * np.arange(17) + 1), rtol=0, atol=1e-16)


@pytest.mark.parametrize("T", [1e-3, 0.3, 1.0, 4.7, 12.0, 29.99, 30.0, 30.01, 45.0, 120.0])
def test_boys_f0_erf(T):
    """F_0(T) = (1/2) sqrt(pi/T) erf(sqrt(T))."""
    F = I.boys(0, T)
    assert abs(F[0] - 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))) < 1e-15


@pytest.mark.parametrize("T", [0.0, 0.5, 2.0, 7.3, 18.0, 29.9, 30.0, 33.0, 60.0])
def test_boys_recursion_identity(T):
    """F_m(T) = (2T F_{m+1}(T) + exp(-T)) / (2m+1) for m < 8."""
    F = I.boys(8, T)
    for m in range(8):
        assert abs(F[m] - (2 * T * F[m + 1] + math.exp(-T)) / (2 * m + 1)) < 1e-15


def test_boys_mpmath_quadrature():
    """F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt by 30-digit mpmath quadrature, m <= 8, T in [0, 60],
    including both sides of the series / asymptotic switch at T = 30: |error| <= 1e-14."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    worst = 0.0
    for T in [0.0, 0.01, 0.5, 1.0, 2.5, 5.0, 9.9, 15.0, 22.2, 29.5, 29.999, 30.0, 30.5, 37.0, 45.0, 60.0]:
        F = I.boys(8, T)
        for m in range(9):
            ref = mp.quad(lambda t: t ** (2 * m) * mp.exp(-T * t * t), [0, 0.5, 1])
            worst = max(worst, abs(F[m] - float(ref)))
    assert worst <= 1e-14, worst


# ----------------------------------------------------------------------------------------- closed forms

def _s_prim(center, a):
    return I.ShellSet(np.array([center]), [0], [np.array([a])], [np.array([1.0])])


def test_closed_form_ss_one_electron():
    """Szabo-Ostlund closed forms for normalised s primitives:
    S = (4ab/p^2)^{3/4} e^{-mu R^2}; T = mu (3 - 2 mu R^2) S; V = -Z (2 pi/p) N_a N_b e^{-mu R^2} F_0(p R_PC^2)."""
    A, B, C = np.array([0.1, -0.3, 0.7]), np.array([1.2, 0.4, -0.5]), np.array([-0.8, 0.9, 1.6])
    a, b, Z = 1.7, 0.35, 3.0
    ss = I.ShellSet(np.array([A, B]), [0, 0], [np.array([a]), np.array([b])], [np.array([1.0]), np.array([1.0])])
    p, mu = a + b, a * b / (a + b)
    R2 = np.sum((A - B) ** 2)
    Na, Nb = (2 * a / math.pi) ** 0.75, (2 * b / math.pi) ** 0.75
    Sab = Na * Nb * (math.pi / p) ** 1.5 * math.exp(-mu * R2)
    Tab = mu * (3 - 2 * mu * R2) * Sab
    P = (a * A + b * B) / p
    T = p * np.sum((P - C) ** 2)
    F0 = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    Vab = -Z * 2 * math.pi / p * Na * Nb * math.exp(-mu * R2) * F0
    Sm, Tm, Vm = ss.overlap(), ss.kinetic(), ss.nuclear(C[None], [Z])
    assert abs(Sm[0, 1] - Sab) < 1e-15 and abs(Sm[0, 0] - 1) < 1e-15
    assert abs(Tm[0, 1] - Tab) < 1e-14
    assert abs(Vm[0, 1] - Vab) < 1e-14


def test_closed_form_ss_eri():
    """(ss|ss) = N_a N_b N_c N_d 2 pi^{5/2} / (p q sqrt(p+q)) e^{-mu_ab R_AB^2} e^{-mu_cd R_CD^2} F_0(rho R_PQ^2)."""
    A, B = np.array([0.0, 0.2, -0.4]), np.array([0.9, -0.6, 0.3])
    C, D = np.array([2.1, 1.0, 0.5]), np.array([1.5, 2.2, -0.8])
    a, b, c, d = 2.3, 0.41, 0.9, 5.5
    s1 = I.ShellSet(np.array([A, B]), [0, 0], [np.array([a]), np.array([b])], [np.array([1.0])] * 2)
    s2 = I.ShellSet(np.array([C, D]), [0, 0], [np.array([c]), np.array([d])], [np.array([1.0])] * 2)
    e = I.eri_block(s1, s2)
    p, q = a + b, c + d
    P, Qc = (a * A + b * B) / p, (c * C + d * D) / q
    rho = p * q / (p + q)
    T = rho * np.sum((P - Qc) ** 2)
    N = np.prod([(2 * x / math.pi) ** 0.75 for x in (a, b, c, d)])
    ref = N * 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * math.exp(-a * b / p * np.sum((A - B) ** 2)) \
        * math.exp(-c * d / q * np.sum((C - D) ** 2)) * 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert abs(e[0, 1, 0, 1] - ref) < 1e-15


# ----------------------------------------------------------------------------------------- quadrature

TINY = [
    (np.array([0.0, 0.0, 0.0]), 1, [1.3, 0.4], [0.7, 0.5]),
    (np.array([0.3, -0.9, 1.1]), 2, [0.9], [1.0]),
    (np.array([-1.0, 0.5, 0.2]), 0, [2.0, 0.3], [0.4, 0.8]),
]


def _oracle_set(shells):
    return I.ShellSet(np.array([s[0] for s in shells]), [s[1] for s in shells],
                      [np.array(s[2]) for s in shells], [np.array(s[3]) for s in shells])


def test_quadrature_overlap_kinetic():
    """S and T (p, d, s shells, contracted) against Gauss-Hermite quadrature; T in gradient form."""
    o, q = _oracle_set(TINY), Q.QShells(TINY)
    assert np.abs(o.overlap() - Q.overlap(q)).max() < 1e-13
    assert np.abs(o.kinetic() - Q.kinetic(q)).max() < 1e-12


def test_quadrature_nuclear():
    """V against quadrature of the Gaussian transform of 1/r, two point charges."""
    o, q = _oracle_set(TINY), Q.QShells(TINY)
    C = np.array([[0.4, 0.4, -0.7], [-1.5, 1.0, 0.9]])
    Z = [8.0, 1.0]
    assert np.abs(o.nuclear(C, Z) - Q.nuclear(q, C, Z)).max() < 1e-11


def test_quadrature_eri_sp_d():
    """(mu nu|lambda sigma) with p/s bra shells and d/s ket shells against quadrature of the
    Gaussian transform of 1/r12 (2D Gauss-Hermite per Cartesian direction)."""
    bra = [TINY[0], TINY[2]]
    ket = [TINY[1], (np.array([0.8, 0.1, -0.6]), 0, [0.6], [1.0])]
    ob, ok = _oracle_set(bra), _oracle_set(ket)
    qb, qk = Q.QShells(bra), Q.QShells(ket)
    e_or = I.eri_block(ob, ok)
    e_q = Q.eri(qb, qk)
    assert np.abs(e_or - e_q).max() < 1e-11


def test_quadrature_eri_dd():
    """A (dd|dd)-containing block, one primitive, against quadrature."""
    sh = [(np.array([0.0, 0.0, 0.0]), 2, [0.7], [1.0]), (np.array([0.5, -0.4, 0.9]), 2, [1.1], [1.0])]
    o, q = _oracle_set(sh[:1]), Q.QShells(sh[:1])
    o2, q2 = _oracle_set(sh[1:]), Q.QShells(sh[1:])
    assert np.abs(I.eri_block(o, o2) - Q.eri(q, q2)).max() < 1e-11


# ----------------------------------------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def dimer():
    return S.water_dimer(0)


@pytest.fixture(scope="module")
def dimer_frags(dimer):
    return Fragments(dimer)


def test_eri_eightfold_symmetry(dimer_frags):
    e = dimer_frags.eri_intra[0]
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.abs(e - e.transpose(perm)).max() < 1e-13
    x = dimer_frags.eri[(0, 1)]
    y = I.eri_block(dimer_frags.shells[1], dimer_frags.shells[0])
    assert np.abs(x - y.transpose(2, 3, 0, 1)).max() < 1e-13


def test_schwarz_and_psd(dimer_frags):
    """The pair-ERI matrix M_(mu nu),(lambda sigma) is positive semidefinite and obeys Schwarz."""
    e = dimer_frags.eri_intra[0]
    n = e.shape[0]
    M = e.reshape(n * n, n * n)
    w = np.linalg.eigvalsh(M)
    assert w.min() > -1e-12 * w.max()
    d = np.sqrt(np.abs(np.diag(M)))
    assert np.all(np.abs(M) <= np.outer(d, d) * (1 + 1e-12) + 1e-15)


def test_unit_self_overlap(dimer_frags):
    for Sm in dimer_frags.S:
        assert np.abs(np.diag(Sm) - 1).max() < 1e-14


def test_translation_invariance(dimer):
    sh0 = I.fragment_shells(dimer, 0)
    shifted = S.System(**{**dimer.__dict__, "xyz": dimer.xyz + np.array([3.3, -1.2, 7.0])})
    sh1 = I.fragment_shells(shifted, 0)
    assert np.abs(sh0.kinetic() - sh1.kinetic()).max() < 1e-12
    C0 = dimer.xyz[3:] / BOHR
    assert np.abs(sh0.nuclear(C0, [8, 1, 1]) - sh1.nuclear(C0 + np.array([3.3, -1.2, 7.0]) / BOHR, [8, 1, 1])).max() < 1e-12
    assert np.abs(I.eri_block(sh0, sh0) - I.eri_block(sh1, sh1)).max() < 1e-12


def _rot_block(system, x, R):
    """AO transformation for s and p shells under a rotation R (p components as a vector)."""
    blocks = []
    for a in system.frag_atoms(x):
        bs = system.basis_sets[system.basis_of_atom[a]]
        for l in bs.l:
            blocks.append(np.eye(1) if l == 0 else R)
    n = sum(b.shape[0] for b in blocks)
    B = np.zeros((n, n))
    i = 0
    for b in blocks:
        B[i:i + b.shape[0], i:i + b.shape[0]] = b
        i += b.shape[0]
    return B


def test_rotation_covariance_sp(dimer):
    """Rotating the molecule by R: s blocks invariant, p blocks transform as vectors, S' = B S B^T."""
    R = S.random_rotation(np.random.default_rng(5))
    rot = S.System(**{**dimer.__dict__, "xyz": dimer.xyz @ R.T})
    s0, s1 = I.fragment_shells(dimer, 0), I.fragment_shells(rot, 0)
    B = _rot_block(dimer, 0, R)
    for f in ("overlap", "kinetic"):
        assert np.abs(B @ getattr(s0, f)() @ B.T - getattr(s1, f)()).max() < 1e-12
    e0, e1 = I.eri_block(s0, s0), I.eri_block(s1, s1)
    e0r = np.einsum("ai,bj,ck,dl,ijkl->abcd", B, B, B, B, e0, optimize=True)
    assert np.abs(e0r - e1).max() < 1e-12


def _ch_fragment(seed=3):
    """A two-atom fragment: C with 3s2p1d, H with 2s (one cation to keep the electron count even)."""
    rng = np.random.default_rng(seed)
    bs = [S.random_basis_set(rng, S.SHELLS_HEAVY_SPD), S.random_basis_set(rng, S.SHELLS_H)]
    return S.System(Z=np.array([6, 1], np.int32), xyz=np.array([[0.0, 0.0, 0.0], [0.7, 0.5, 0.6]]),
                    frag_of_atom=np.array([0, 0], np.int32), charge=np.array([1], np.int32),
                    basis_of_atom=np.array([0, 1], np.int32), basis_sets=bs)


def test_rotation_invariants_with_d():
    """With d shells (Cartesian d blocks do not transform orthogonally): the generalised eigenvalues
    of (T, S) and (h, S), of the pair-ERI matrix in the S (x) S metric, and the isolated RHF energy
    are invariant under a rigid rotation."""
    import scipy.linalg
    sysd = _ch_fragment()
    R = S.random_rotation(np.random.default_rng(11))
    rot = S.System(**{**sysd.__dict__, "xyz": sysd.xyz @ R.T})
    f0, f1 = Fragments(sysd), Fragments(rot)
    for mat in ("T", "h"):
        a = scipy.linalg.eigh(getattr(f0, mat)[0], f0.S[0], eigvals_only=True)
        b = scipy.linalg.eigh(getattr(f1, mat)[0], f1.S[0], eigvals_only=True)
        assert np.abs(a - b).max() < 1e-11 * np.abs(a).max()
    n = f0.n_ao[0]
    w = []
    for f in (f0, f1):
        SS = np.kron(f.S[0], f.S[0])
        w.append(scipy.linalg.eigh(f.eri_intra[0].reshape(n * n, n * n), SS + 1e-300, eigvals_only=True,
                                   subset_by_index=[n * n - 40, n * n - 1]))
    assert np.abs(w[0] - w[1]).max() < 1e-9 * np.abs(w[0]).max()
    e0 = f0.rhf(0, np.zeros((n, n)))[2]
    e1 = f1.rhf(0, np.zeros((n, n)))[2]
    assert abs(e0 - e1) < 1e-9


# ----------------------------------------------------------------------------------------- multipole limits

def test_ss_far_limit():
    """Two same-centre s-shell pairs far apart: (ab|cd) R -> S_ab S_cd (charge-charge limit)."""
    sa = I.ShellSet(np.zeros((2, 3)), [0, 0], [np.array([1.1, 0.3]), np.array([0.5, 2.0])],
                    [np.array([0.6, 0.8]), np.array([0.9, 0.4])])
    for R in (40.0, 90.0):
        sb = I.ShellSet(np.array([[0, 0, R], [0, 0, R]]), [0, 0], [np.array([0.7, 0.2]), np.array([3.0, 0.8])],
                        [np.array([0.5, 0.5]), np.array([0.3, 0.9])])
        e = I.eri_block(sa, sb)
        Sa, Sb = sa.overlap(), sb.overlap()
        assert abs(e[0, 1, 0, 1] * R - Sa[0, 1] * Sb[0, 1]) < 1e-13


def test_water_pair_dipole_limit(dimer):
    """E_xy of two neutral fragments with frozen isolated densities, translated apart along n:
    E_xy -> dipole-dipole (mu_x.mu_y - 3 (mu_x.n)(mu_y.n)) / R^3, with the residual falling as R^-4.
    Dipoles come from quadrature dipole integrals (tests/quadrature.py), not from the oracle."""
    base = Fragments(dimer, inter=False)
    D = base.isolated()
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    mus = []
    for x in range(2):
        atoms = dimer.frag_atoms(x)
        cen = (dimer.Z[atoms][:, None] * dimer.xyz[atoms]).sum(0) / dimer.Z[atoms].sum() / BOHR
        shells = []
        for a in atoms:
            bs = dimer.basis_sets[dimer.basis_of_atom[a]]
            for l, e, c in zip(bs.l, bs.exps, bs.coefs):
                shells.append((dimer.xyz[a] / BOHR, l, e, c))
        M = Q.dipole(Q.QShells(shells), origin=cen)
        nuc = (dimer.Z[atoms][:, None] * (dimer.xyz[atoms] / BOHR - cen)).sum(0)
        mus.append(nuc - np.einsum("kij,ij->k", M, D[x]))
    scaled = []
    for R in (60.0, 120.0, 240.0):
        moved = dimer.xyz.copy()
        c0 = (dimer.Z[:3, None] * dimer.xyz[:3]).sum(0) / 10
        c1 = (dimer.Z[3:, None] * dimer.xyz[3:]).sum(0) / 10
        moved[3:] += (c0 - c1) + n * R * BOHR
        fr = Fragments(S.System(**{**dimer.__dict__, "xyz": moved}))
        Exy = fr.energies(D)["E_pair"][(0, 1)]
        Edd = (mus[0] @ mus[1] - 3 * (mus[0] @ n) * (mus[1] @ n)) / R ** 3
        assert abs(Exy - Edd) < 0.25 * abs(Edd)
        scaled.append((Exy - Edd) * R ** 4)
    # the residual is the dipole-quadrupole term: (E_xy - E_dd) R^4 is constant up to O(1/R)
    assert abs(scaled[1] / scaled[0] - 1) < 0.01 and abs(scaled[2] / scaled[1] - 1) < 0.005


# ----------------------------------------------------------------------------------------- SCF / FEF

def test_config0_density_is_valid(dimer_frags):
    """D = 2 C C^T with C = G (G^T S G)^{-1/2}: tr(DS) = N_e and D S D = 2 D."""
    for x in range(2):
        G = S.random_orbital_coefficients(100 + x, dimer_frags.n_ao[x], 5)
        D = orthonormal_density(G, dimer_frags.S[x])
        assert abs(np.trace(D @ dimer_frags.S[x]) - 10) < 1e-12
        assert np.abs(D @ dimer_frags.S[x] @ D - 2 * D).max() < 1e-12


def test_isolated_rhf_invariants(dimer_frags):
    """Isolated-fragment RHF: tr(DS) = N_e, DSD = 2D, FDS - SDF = 0, and the orbital energies
    from the oracle's orthogonalised problem equal scipy's generalised symmetric eigensolver."""
    import scipy.linalg
    D = dimer_frags.isolated()
    for x in range(2):
        Sx = dimer_frags.S[x]
        F = dimer_frags.h[x] + dimer_frags.G(x, D[x])
        assert abs(np.trace(D[x] @ Sx) - 10) < 1e-10
        assert np.abs(D[x] @ Sx @ D[x] - 2 * D[x]).max() < 1e-10
        assert np.abs(F @ D[x] @ Sx - Sx @ D[x] @ F).max() < 1e-8
        X = dimer_frags.X[x]
        if X.shape[1] == Sx.shape[0]:
            e1 = np.linalg.eigvalsh(X.T @ F @ X)
            e2 = scipy.linalg.eigh(F, Sx, eigvals_only=True)
            assert np.abs(e1 - e2).max() < 1e-9


def test_canonical_orthogonaliser_drops_dependence():
    """X^T S X = 1, and an exactly duplicated function is dropped."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((6, 6))
    Sm = A @ A.T + 6 * np.eye(6)
    Sd = np.block([[Sm, Sm[:, :1]], [Sm[:1, :], Sm[:1, :1]]])
    X = canonical_orthogonaliser(Sd)
    assert X.shape == (7, 6)
    assert np.abs(X.T @ Sd @ X - np.eye(6)).max() < 1e-12


@pytest.fixture(scope="module")
def dimer_solution(dimer_frags):
    return dimer_frags.solve(e_tol=1e-11)


def test_fef_fixed_point_commutators(dimer_frags, dimer_solution):
    """At the FEF fixed point every fragment's full F^x = h + G + omega commutes with D^x in the S metric."""
    D = dimer_solution["D"]
    F = dimer_frags.fock(D)
    for x in range(2):
        Sx = dimer_frags.S[x]
        assert np.abs(F[x] @ D[x] @ Sx - Sx @ D[x] @ F[x]).max() < 1e-7


def test_energy_partition_sums(dimer_frags, dimer_solution):
    En = dimer_solution["energies"]
    assert abs(En["E_x"].sum() - En["E_tot"]) < 1e-10


def test_pair_coulomb_symmetry(dimer_frags, dimer_solution):
    """tr(D^x J[D^y]) = tr(D^y J[D^x]), built from the ERI blocks computed in each order."""
    from oracle.fef import coulomb
    D = dimer_solution["D"]
    e01 = dimer_frags.eri[(0, 1)]
    e10 = I.eri_block(dimer_frags.shells[1], dimer_frags.shells[0])
    assert abs(np.sum(D[0] * coulomb(e01, D[1])) - np.sum(D[1] * coulomb(e10, D[0]))) < 1e-11


def test_total_energy_stationary(dimer_frags, dimer_solution):
    """E_tot is stationary at the fixed point (F^x = dE_tot/dD^x): an occupied-virtual rotation by
    kappa changes E_tot by O(kappa^2)."""
    D = dimer_solution["D"]
    F = dimer_frags.fock(D)
    E0 = dimer_frags.energies(D)["E_tot"]
    x = 0
    X = dimer_frags.X[x]
    eps, Cp = np.linalg.eigh(X.T @ F[x] @ X)
    C = X @ Cp
    nocc = 5

    def rotated(k):
        Cn = C.copy()
        i, a = nocc - 1, nocc + 1
        Cn[:, i] = math.cos(k) * C[:, i] + math.sin(k) * C[:, a]
        Dn = [d.copy() for d in D]
        Dn[x] = 2 * Cn[:, :nocc] @ Cn[:, :nocc].T
        return dimer_frags.energies(Dn)["E_tot"] - E0

    d1, d2 = rotated(1e-3), rotated(2e-3)
    assert abs(d1) < 1e-4
    assert 3.6 < d2 / d1 < 4.4


def test_single_fragment_is_plain_rhf():
    """One fragment (or a cutoff that keeps no pair): FEF reduces to the fragment's own RHF."""
    sysm = S.water_dimer(1, r_oo=3.0)
    fr = Fragments(sysm, cutoff_A=0.1)
    assert fr.pairs == []
    res = fr.solve(e_tol=1e-10)
    iso = fr.isolated()
    for x in range(2):
        assert np.abs(res["D"][x] - iso[x]).max() < 1e-8
    assert res["n_macro"] == 1


# ----------------------------------------------------------------------------------------- warm-start network

def test_mlp_oracle_gradient_finite_differences():
    """The oracle MLP's analytic gradient against central finite differences of its loss."""
    from oracle import mlp
    rng = np.random.default_rng(3)
    n_in, n_h, n_out = 5, 7, 4
    n_par = sum(int(np.prod(s)) for s in mlp.shapes(n_in, n_h, n_out))
    theta = rng.standard_normal(n_par) * 0.4
    X = rng.standard_normal((9, n_in))
    T = rng.standard_normal((9, n_out))
    L, g = mlp.loss_and_grad(theta, X, T, n_in, n_h, n_out)
    h = 1e-6
    for i in rng.choice(n_par, 25, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, T, n_in, n_h, n_out)[0] - mlp.loss_and_grad(tm, X, T, n_in, n_h, n_out)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-8 * max(1.0, abs(fd))
    assert abs(L - np.mean((mlp.forward(theta, X, n_in, n_h, n_out)[0] - T) ** 2)) < 1e-14


# ------------------------------------------------------------------------------------- E_M2

def _second_order_by_determinants(eri_mo, eps, nocc):
    """Second-order Rayleigh-Schroedinger energy with the Moller-Plesset partition, summed over
    doubly excited Slater determinants in the spin-orbital basis: E2 = sum_{i<j, a<b} |<ij||ab>|^2 /
    (e_i + e_j - e_a - e_b), <pq||rs> = <pq|rs> - <pq|sr> from the spatial (pr|qs) and spin
    orthogonality (Slater-Condon rules for a double excitation)."""
    n = len(eps)
    so = [(p, s) for p in range(n) for s in (0, 1)]
    occ = [k for k, (p, s) in enumerate(so) if p < nocc]
    vir = [k for k, (p, s) in enumerate(so) if p >= nocc]

    def phys(k1, k2, k3, k4):  # <k1 k2|k3 k4>
        (p, a), (q, b), (r, c), (t, d) = so[k1], so[k2], so[k3], so[k4]
        return eri_mo[p, r, q, t] if (a == c and b == d) else 0.0

    e2 = 0.0
    for ii, i in enumerate(occ):
        for j in occ[ii + 1:]:
            for aa, a in enumerate(vir):
                for b in vir[aa + 1:]:
                    v = phys(i, j, a, b) - phys(i, j, b, a)
                    e2 += v * v / (eps[so[i][0]] + eps[so[j][0]] - eps[so[a][0]] - eps[so[b][0]])
    return e2


def test_e_m2_equals_determinant_second_order(dimer_frags, dimer_solution):
    """The oracle's closed-shell E_M2 of each fragment (in its FEF field) equals the second-order
    energy summed over spin-orbital double excitations with antisymmetrised integrals (an
    independent route that fixes the exchange term and the factor of 2)."""
    ref = dimer_frags
    D = dimer_solution["D"]
    F = ref.fock(D)
    for x in range(ref.nf):
        X = ref.X[x]
        eps, Cp = np.linalg.eigh(X.T @ F[x] @ X)
        C = X @ Cp
        eri = I.eri_block(ref.shells[x], ref.shells[x])
        eri_mo = np.einsum("mp,nq,mnls,lr,st->pqrt", C, C, eri, C, C, optimize=True)
        e_det = _second_order_by_determinants(eri_mo, eps, ref.n_occ[x])
        e_m2 = ref.e_m2(x, F[x])
        assert e_m2 < 0.0
        assert abs(e_m2 - e_det) < 1e-12 * max(1.0, abs(e_det)), (x, e_m2, e_det)


def test_e_m2_orbital_rotation_invariance(dimer_frags, dimer_solution):
    """E_M2 depends on the occupied and virtual spaces and the canonical energies only: a random
    orthogonal change of the fragment's AO basis (applied to S, F and the orbitals) leaves it
    unchanged, checked here through the rotation of the whole fragment in space (p and d blocks
    rotate with the geometry)."""
    ref = dimer_frags
    D = dimer_solution["D"]
    F = ref.fock(D)
    e0 = ref.e_m2(0, F[0])
    sysm = ref.system
    R = S.random_rotation(np.random.default_rng(7))
    at = sysm.frag_atoms(0)
    moved = S.System(Z=sysm.Z[at], xyz=(sysm.xyz[at] - sysm.xyz[at].mean(0)) @ R.T, frag_of_atom=np.zeros(len(at), np.int32),
                     charge=np.zeros(1, np.int32), basis_of_atom=sysm.basis_of_atom[at], basis_sets=sysm.basis_sets)
    iso = Fragments(moved, inter=False)
    iso0 = Fragments(S.System(Z=sysm.Z[at], xyz=sysm.xyz[at], frag_of_atom=np.zeros(len(at), np.int32),
                              charge=np.zeros(1, np.int32), basis_of_atom=sysm.basis_of_atom[at],
                              basis_sets=sysm.basis_sets), inter=False)
    Da, Fa, *_ = iso0.rhf(0, np.zeros_like(iso0.S[0]), e_tol=1e-13, comm_tol=1e-11)
    Db, Fb, *_ = iso.rhf(0, np.zeros_like(iso.S[0]), e_tol=1e-13, comm_tol=1e-11)
    assert abs(iso0.e_m2(0, Fa) - iso.e_m2(0, Fb)) < 1e-10
    assert e0 < 0.0


# ------------------------------------------------------------------------------------- E_D2

def test_e_d2_equals_spin_orbital_sum(dimer_frags, dimer_solution):
    """The oracle's E_D2 of the dimer equals the second-order sum over spin-orbital double excitations
    with one electron excited on each fragment, <Phi_{i s -> a s, j t -> b t}|V_xy|Phi_0> = (ia|jb) for
    every spin pair (s, t) and no exchange between fragments (an independent route that fixes the
    spin factor 4 and the absence of an exchange term)."""
    ref = dimer_frags
    D = dimer_solution["D"]
    F = ref.fock(D)
    Cx, ex = ref.canonical_orbitals(0, F[0])
    Cy, ey = ref.canonical_orbitals(1, F[1])
    ox, oy = ref.n_occ
    eri = I.eri_block(ref.shells[0], ref.shells[1])
    mo = np.einsum("mp,nq,mnls,lr,st->pqrt", Cx, Cx, eri, Cy, Cy, optimize=True)
    e2 = 0.0
    for i in range(ox):
        for a in range(ox, len(ex)):
            for j in range(oy):
                for b in range(oy, len(ey)):
                    for s in (0, 1):
                        for t in (0, 1):
                            v = mo[i, a, j, b]  # spin s on x, spin t on y: a direct Coulomb element
                            e2 += v * v / (ex[i] + ey[j] - ex[a] - ey[b])
    e_d2 = ref.e_d2(0, 1, F[0], F[1])
    assert e_d2 < 0.0
    assert abs(e_d2 - e2) < 1e-13 * max(1.0, abs(e2))


def test_e_d2_far_field_r6():
    """Far apart, the dimer second-order term of two neutral fragments is dispersion-like: with frozen
    isolated orbitals E_D2(R) falls as R^-6 (dipole-dipole transitions); the local slope
    d ln|E| / d ln R between 30 and 60 bohr is -6 within 1 %."""
    base = S.water_dimer(0)
    at1 = base.frag_atoms(1)
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    vals = []
    for R in (30.0, 60.0):
        xyz = base.xyz.copy()
        shift = R * BOHR * u - (xyz[at1].mean(0) - xyz[base.frag_atoms(0)].mean(0))
        xyz[at1] += shift
        sysm = S.System(Z=base.Z, xyz=xyz, frag_of_atom=base.frag_of_atom, charge=base.charge,
                        basis_of_atom=base.basis_of_atom, basis_sets=base.basis_sets)
        ref = Fragments(sysm, inter=False)
        F = []
        for x in range(2):
            Dx, Fx, *_ = ref.rhf(x, np.zeros_like(ref.S[x]), e_tol=1e-13, comm_tol=1e-11)
            F.append(Fx)
        vals.append(ref.e_d2(0, 1, F[0], F[1]))
    slope = math.log(abs(vals[1]) / abs(vals[0])) / math.log(2.0)
    assert vals[0] < 0 and vals[1] < 0
    assert abs(slope + 6.0) < 0.06, slope


# ------------------------------------------------------------------------------------- far field

def _dimer_at(R_bohr):
    base = S.water_dimer(0)
    at0, at1 = base.frag_atoms(0), base.frag_atoms(1)
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    xyz = base.xyz.copy()
    xyz[at1] += R_bohr * BOHR * u - (xyz[at1].mean(0) - xyz[at0].mean(0))
    return S.System(Z=base.Z, xyz=xyz, frag_of_atom=base.frag_of_atom, charge=base.charge,
                    basis_of_atom=base.basis_of_atom, basis_sets=base.basis_sets)


def test_moment_integrals_pins():
    """<mu|1|nu> = S; the dipole integrals follow a shift of the expansion point, <r - c'> = <r - c> +
    (c - c') S; the second moments are symmetric and positive on the diagonal."""
    ref = Fragments(_dimer_at(8.0), far_field=True)
    M = ref.M[0]
    assert np.abs(M[0] - ref.S[0]).max() < 1e-14
    t = np.array([0.3, -0.2, 0.5])
    M2 = ref.shells[0].moments(ref.centre[0] + t)
    assert np.abs(M2[1:4] - (M[1:4] - t[:, None, None] * M[0])).max() < 1e-13
    for k in (4, 7, 9):
        assert (np.diag(M[k]) > 0).all()
    assert np.abs(M - M.transpose(0, 2, 1)).max() < 1e-13


def test_far_field_energy_against_exact_pair():
    """Two waters far apart, frozen isolated densities: the multipole pair energy (charges, dipoles,
    second moments of nuclei + electrons) approaches the exact E_xy (exact V and J integrals); the
    first terms it leaves out (dipole-octupole) fall as R^-5, so the error drops by more than 2^4.5
    from 20 to 40 bohr, where it is below 5 % and 1 % of the interaction."""
    errs = []
    for R in (20.0, 40.0):
        sysm = _dimer_at(R)
        exact = Fragments(sysm)                                  # all pairs near: exact V + J
        far = Fragments(sysm, cutoff_A=0.5, far_field=True)      # the pair is beyond the cutoff
        D = []
        for x in range(2):
            Dx, *_ = exact.rhf(x, np.zeros_like(exact.S[x]), e_tol=1e-13, comm_tol=1e-11)
            D.append(Dx)
        e_exact = exact.energies(D)["E_pair"][(0, 1)]
        e_far = far.energies(D)["E_pair"][(0, 1)]
        assert abs(e_far - e_exact) < (0.05 if R < 30 else 0.01) * abs(e_exact), (R, e_far, e_exact)
        errs.append(abs(e_far - e_exact))
    assert errs[1] < errs[0] / 2 ** 4.5, errs


def test_far_field_recovers_cluster_truncation():
    """A 24-water cluster (8.9 A cube, 1 g/cm^3) at a 5 A pair cutoff, frozen isolated densities:
    the paper's sum over every other fragment (all pairs exact) fixes E_tot.  The plain cutoff misses more than
    1 mEh of it (158 of 276 pairs dropped); with the multipole far field for those pairs the miss is
    below 5 % of that."""
    system = S.water_box(24, seed=1)
    exact = Fragments(system, schwarz=1e-12)
    D = exact.isolated()
    e_all = exact.energies(D)["E_tot"]
    e_cut = Fragments(system, cutoff_A=5.0, schwarz=1e-12).energies(D)["E_tot"]
    far = Fragments(system, cutoff_A=5.0, schwarz=1e-12, far_field=True)
    assert len(far.far_pairs) > 100
    e_far = far.energies(D)["E_tot"]
    assert abs(e_cut - e_all) > 1e-3
    assert abs(e_far - e_all) < 0.05 * abs(e_cut - e_all), (e_cut - e_all, e_far - e_all)


def test_far_field_fock_is_energy_derivative():
    """omega_far of fragment x is the derivative of the far-field energy with respect to D^x:
    central differences along a random symmetric direction agree with tr(Delta omega_far)."""
    ref = Fragments(_dimer_at(12.0), cutoff_A=0.5, far_field=True)
    rng = np.random.default_rng(3)
    D = [orthonormal_density(S.random_orbital_coefficients(50 + x, ref.n_ao[x], ref.n_occ[x]), ref.S[x])
         for x in range(2)]
    om, _ = ref.far_terms(D)
    for x in range(2):
        A = rng.standard_normal(D[x].shape)
        Dl = (A + A.T) / 2
        h = 1e-4
        Dp = [d.copy() for d in D]
        Dm = [d.copy() for d in D]
        Dp[x] += h * Dl
        Dm[x] -= h * Dl
        ep = sum(ref.far_terms(Dp)[1].values())
        em = sum(ref.far_terms(Dm)[1].values())
        assert abs((ep - em) / (2 * h) - np.sum(Dl * om[x])) < 1e-8


# ----------------------------------------------------------------------------------------- screening and pairs
# The sum over y != x of Eq. wc / Eq. dp2e is cut at a fragment-pair cutoff and the shell quartets
# are screened by the Schwarz bound (both readings of the configurations): these pins fix the
# oracle's screening factors, quartet counts and pair list by brute force.

def _shell_ranges(ls):
    out, k = [], 0
    for l in ls:
        n = (l + 1) * (l + 2) // 2
        out.append(range(k, k + n))
        k += n
    return out


def _schwarz_from_diagonal(diag, ls):
    """Q_ab = sqrt(max_{mu in a, nu in b} |(mu nu|mu nu)|) from the AO-pair diagonal (n, n)."""
    r = _shell_ranges(ls)
    return np.array([[math.sqrt(np.abs(diag[np.ix_(ra, rb)]).max()) for rb in r] for ra in r])


def test_schwarz_factors_against_quadrature():
    """or_schwarz on contracted s, p and d shells: Q_ab from the diagonal ERIs (mu nu|mu nu) computed
    by brute-force quadrature of the Gaussian transform of 1/r12, independent of the Obara-Saika code."""
    o, q = _oracle_set(TINY), Q.QShells(TINY)
    Qo = o.schwarz()
    Qq = _schwarz_from_diagonal(Q.eri_diagonal(q), [s[1] for s in TINY])
    assert Qo.shape == (3, 3)
    assert np.abs(Qo - Qo.T).max() == 0.0
    assert np.abs(Qo - Qq).max() < 1e-11 * Qq.max()


def _spd_dimer(seed=3, r=3.1):
    """Two water-like fragments whose oxygen carries s, p and d shells (a d-shell fragment)."""
    rb, rg = S._streams(seed, 2)
    bs = [S.random_basis_set(rb, S.SHELLS_HEAVY_SPD), S.random_basis_set(rb, S.SHELLS_H)]
    z, w = S.water_geometry()
    u = S.random_unit(rg)
    frags = [(z, w @ S.random_rotation(rg).T + k * r * u) for k in range(2)]
    return S._assemble(frags, bs, [np.array([0, 1, 1])] * 2, "spd dimer")


@pytest.fixture(scope="module")
def spd_pair():
    system = _spd_dimer()
    sh = [I.fragment_shells(system, x) for x in range(2)]
    full = {k: I.eri_block(sh[k[0]], sh[k[1]]) for k in [(0, 0), (1, 1), (0, 1)]}
    return sh, full


def test_schwarz_factors_d_fragment(spd_pair):
    """or_schwarz of a fragment with d shells equals sqrt of the largest diagonal element of each
    shell pair's block, taken by brute force from the full (unscreened) ERI tensor."""
    sh, full = spd_pair
    for k in range(2):
        n = sh[k].n_ao
        diag = np.einsum("ijij->ij", full[(k, k)].reshape(n, n, n, n))
        Qb = _schwarz_from_diagonal(diag, list(sh[k].l))
        assert np.abs(sh[k].schwarz() - Qb).max() < 1e-14 * Qb.max()


def test_packed_coulomb_exchange_tensor(spd_pair):
    """The pair-packed Coulomb-minus-half-exchange tensor that the GPU keeps per fragment,
    CT[rs][pq] = C[pq][rs] + [la != si] C[pq][(si la)] with C[mn][ls] = (mn|ls) - (ml|ns)/2 over
    pairs mu <= nu and la <= si (row-major upper triangle), gives G[D] = J[D] - K[D]/2 as one product
    G_pq = sum_rs CT[rs][pq] D_rs for a symmetric D (against the oracle's plain J and K), and it
    factorises as CT[rs][pq] = Cs[pq][rs] w_rs with Cs symmetric (w = 1 for la != si, 1/2 for
    la = si): the identity that lets one triangle of Cs hold the whole tensor."""
    from oracle.fef import coulomb, exchange
    sh, full = spd_pair
    n = sh[0].n_ao
    eri = full[(0, 0)].reshape(n, n, n, n)
    iu = np.triu_indices(n)
    C = eri - 0.5 * eri.transpose(0, 2, 1, 3)
    rows = C[iu[0], iu[1]]                 # C[pq][l, s]
    Cpk = rows[:, iu[0], iu[1]]            # C[pq][rs]
    Cswap = rows[:, iu[1], iu[0]]          # C[pq][(si la)]
    off = (iu[0] != iu[1]).astype(np.float64)
    CT = (Cpk + off[None, :] * Cswap).T    # CT[rs][pq]
    rng = np.random.default_rng(11)
    A = rng.standard_normal((n, n))
    D = A + A.T
    G_ref = coulomb(eri, D) - 0.5 * exchange(eri, D)
    G_pk = CT.T @ D[iu]
    assert np.abs(G_pk - G_ref[iu]).max() <= 1e-12 * np.abs(G_ref).max()
    Cs = Cpk + Cswap
    w = np.where(off > 0, 1.0, 0.5)
    assert np.abs(CT - (Cs * w[None, :]).T).max() <= 1e-14 * np.abs(CT).max()
    assert np.abs(Cs - Cs.T).max() <= 1e-13 * np.abs(Cs).max()


def test_quartet_count_brute_force(spd_pair):
    """or_count_quartets equals a brute-force count over all a <= b in x, c <= d in y of
    Q_ab Q_cd >= tau, a quartet whose product equals tau is kept, and every dropped quartet has
    max |(ab|cd)| <= Q_ab Q_cd < tau (Schwarz inequality), zeroed by the screened ERI block."""
    sh, full = spd_pair
    Qx, Qy = sh[0].schwarz(), sh[1].schwarz()
    rx, ry = _shell_ranges(list(sh[0].l)), _shell_ranges(list(sh[1].l))
    quartets = [(a, b, c, d) for a in range(sh[0].n_sh) for b in range(a, sh[0].n_sh)
                for c in range(sh[1].n_sh) for d in range(c, sh[1].n_sh)]
    prods = np.array([Qx[a, b] * Qy[c, d] for a, b, c, d in quartets])
    assert len(quartets) == (10 * 11 // 2) * (10 * 11 // 2)
    tie = float(np.sort(prods)[len(prods) // 3])
    for tau in [0.0, 1e-12, 1e-6, float(np.median(prods)), tie, np.nextafter(tie, np.inf), 2 * prods.max()]:
        brute = int(sum(1 for p in prods if p >= tau))
        assert I.count_quartets(sh[0], sh[1], Qx, Qy, tau) == brute, tau
    assert I.count_quartets(sh[0], sh[1], Qx, Qy, tie) == I.count_quartets(sh[0], sh[1], Qx, Qy,
                                                                          np.nextafter(tie, np.inf)) + \
        int(np.sum(prods == tie))
    tau = float(np.median(prods))
    e_full = full[(0, 1)]
    e_scr = I.eri_block(sh[0], sh[1], Qx, Qy, tau)
    n_dropped = 0
    for a in range(sh[0].n_sh):
        for b in range(sh[0].n_sh):
            for c in range(sh[1].n_sh):
                for d in range(sh[1].n_sh):
                    blk = np.ix_(rx[a], rx[b], ry[c], ry[d])
                    if Qx[a, b] * Qy[c, d] < tau:
                        n_dropped += 1
                        assert np.abs(e_full[blk]).max() <= Qx[a, b] * Qy[c, d] * (1 + 1e-12) + 1e-300
                        assert not np.any(e_scr[blk])
                    else:
                        assert np.array_equal(e_scr[blk], e_full[blk])
    assert n_dropped > 0


def _hand_placed_clusters():
    """Two-atom fragments along the axes, so that inter-fragment distances are exact doubles:
    the closest atoms of fragments 0 and 1 are 8 - 1e-9 A apart (second atom of 0, first of 1),
    of fragments 0 and 2 exactly 8 A, of fragments 1 and 3 8 + 1e-9 A, of fragments 2 and 3
    8 - 1e-9 A; every other pair is farther than 8 A apart."""
    e = 1e-9
    xyz = np.array([
        [0.0, 0.0, 0.0], [-0.74, 0.0, 0.0],                  # fragment 0
        [8.0 - e, 0.0, 0.0], [8.0 - e + 0.74, 0.0, 0.0],      # fragment 1
        [-0.74, 0.0, -8.0], [-0.74, -0.74, -8.0],              # fragment 2
        [8.0 - e + 0.74, 0.0, 8.0 + e], [-0.74, -0.74, -16.0 + e],  # fragment 3
    ])
    bs = S.random_basis_set(np.random.default_rng(0), S.SHELLS_H)
    return S.System(Z=np.ones(8, np.int32), xyz=xyz, frag_of_atom=np.repeat(np.arange(4), 2).astype(np.int32),
                    charge=np.zeros(4, np.int32), basis_of_atom=np.zeros(8, np.int32), basis_sets=[bs],
                    name="hand-placed pairs")


HAND_PLACED_PAIRS_8A = [(0, 1), (2, 3)]


def test_neighbour_pairs_hand_placed():
    """Fragments.neighbour_pairs keeps (x < y) exactly when the minimum inter-fragment atom-atom
    distance is below the cutoff: against the hand-placed set and an explicit loop over all atoms."""
    import types
    system = _hand_placed_clusters()
    atoms = [system.frag_atoms(x) for x in range(system.n_frag)]
    host = types.SimpleNamespace(system=system, nf=system.n_frag, atoms=atoms)
    got = Fragments.neighbour_pairs(host, 8.0)
    assert got == HAND_PLACED_PAIRS_8A
    brute = []
    for x in range(system.n_frag):
        for y in range(x + 1, system.n_frag):
            dmin = min(math.dist(system.xyz[i], system.xyz[j]) for i in atoms[x] for j in atoms[y])
            if dmin < 8.0:
                brute.append((x, y))
    assert got == brute
    assert Fragments.neighbour_pairs(host, 8.0 + 2e-9) == [(0, 1), (0, 2), (1, 3), (2, 3)]
    assert Fragments.neighbour_pairs(host, 8.0 - 5e-10) == [(0, 1), (2, 3)]
    assert Fragments.neighbour_pairs(host, 8.0 + 5e-10) == [(0, 1), (0, 2), (2, 3)]
    assert Fragments.neighbour_pairs(host, None) == [(x, y) for x in range(4) for y in range(x + 1, 4)]
    assert Fragments.neighbour_pairs(host, 1.0) == []
