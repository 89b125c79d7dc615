"""CPU oracle: the fragment-effective-field (FEF) mean field, plain NumPy in FP64.

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the CPU-baseline leg of the
benchmark may import this module.  It shares no code with the CUDA library.

Follows the paper's Theory section, "Fragment Mean Field":

* product ansatz with the antisymmetriser dropped (Eq. prodspace): each fragment x has its own
  determinant in its own monomer-centred AO basis, and there is no inter-fragment exchange;
* the polarisation-screened fragment Fock matrix F~ = h(1) + (2J - K) + omega_x; in AO form with
  D = 2 C_occ C_occ^T this is F^x = h^x + G[D^x] + omega_x with G[D] = J[D] - K[D]/2;
* omega_x = h~ + 2 v (Eq. wc): h~ is the attraction of x's electrons to the nuclei of every other
  fragment (equation after Eq. wc) and 2 v^{mu j}_{nu j} with v from Eq. dp2e equals the Coulomb
  matrix J[D^y] of each other fragment's density, J[D^y]_{mu nu} = sum_{lambda sigma in y}
  (mu nu|lambda sigma) D^y_{lambda sigma};
* the field is relaxed to all orders (the polarisation-screened mean field): every fragment's RHF
  is solved in the field of the others and the field is rebuilt until all fragments are
  self-consistent;
* energies from the reference expectation values <H_x> and <H_xy> of the Hamiltonian partition
  (Eqs. NHx, NHxy, clusterH), with pairs counted once.

Readings of points the paper leaves open (units bohr/hartree, h(1) with own nuclei only, the
cutoff dropping J and V of a fragment together, Schwarz screening at shell level, unordered pair
sums, canonical orthogonalisation, nested macro/micro iteration) are the ones listed in the design
notes of this repository.
"""
from __future__ import annotations

import math

import numpy as np

from synth.systems import ANGSTROM_PER_BOHR, frag_n_occ
from . import integrals as I


def canonical_orthogonaliser(S: np.ndarray, s_min: float = 1e-7) -> np.ndarray:
    """X = U s^{-1/2} over eigenvalues s >= s_min of S, so that X^T S X = 1."""
    s, U = np.linalg.eigh(S)
    keep = s >= s_min
    return U[:, keep] / np.sqrt(s[keep])


def density_from_orbitals(C_occ: np.ndarray) -> np.ndarray:
    return 2.0 * C_occ @ C_occ.T


def orthonormal_density(G: np.ndarray, S: np.ndarray) -> np.ndarray:
    """D = 2 C C^T with C = G (G^T S G)^{-1/2}, i.e. occupied orbitals orthonormal in the S metric."""
    M = G.T @ S @ G
    w, V = np.linalg.eigh(M)
    C = G @ (V / np.sqrt(w)) @ V.T
    return density_from_orbitals(C)


def coulomb(eri: np.ndarray, D: np.ndarray) -> np.ndarray:
    """J[D]_{mu nu} = sum_{lambda sigma} (mu nu|lambda sigma) D_{lambda sigma}."""
    n1 = eri.shape[0]
    return (eri.reshape(n1 * n1, -1) @ D.ravel()).reshape(n1, n1)


def exchange(eri: np.ndarray, D: np.ndarray) -> np.ndarray:
    """K[D]_{mu nu} = sum_{lambda sigma} (mu lambda|nu sigma) D_{lambda sigma}."""
    return np.einsum("mlns,ls->mn", eri, D, optimize=True)


def nuclear_repulsion(Z1, R1, Z2=None, R2=None) -> float:
    """sum over distinct nucleus pairs Z_A Z_B / R_AB (within one set, or between two sets)."""
    if Z2 is None:
        e = 0.0
        for a in range(len(Z1)):
            for b in range(a):
                e += Z1[a] * Z1[b] / np.linalg.norm(R1[a] - R1[b])
        return e
    e = 0.0
    for a in range(len(Z1)):
        for b in range(len(Z2)):
            e += Z1[a] * Z2[b] / np.linalg.norm(R1[a] - R2[b])
    return e


class Fragments:
    """All integrals of a fragmented system the FEF mean field needs, held in memory.

    cutoff_A: fragment pairs whose minimum inter-fragment atom-atom distance is not below the
    cutoff are dropped (both J and V).  None keeps all pairs.
    schwarz: shell quartets with Q_ab Q_cd < schwarz are dropped (0 keeps all).
    """

    def __init__(self, system, cutoff_A: float | None = None, schwarz: float = 0.0, inter: bool = True,
                 far_field: bool = False):
        self.system = system
        self.nf = system.n_frag
        self.schwarz_tau = schwarz
        self.shells = [I.fragment_shells(system, x) for x in range(self.nf)]
        self.n_ao = [s.n_ao for s in self.shells]
        self.n_occ = [frag_n_occ(system, x) for x in range(self.nf)]
        self.atoms = [system.frag_atoms(x) for x in range(self.nf)]
        self.Zn = [system.Z[a].astype(np.float64) for a in self.atoms]
        self.Rn = [system.xyz[a] / ANGSTROM_PER_BOHR for a in self.atoms]
        self.S = [s.overlap() for s in self.shells]
        self.T = [s.kinetic() for s in self.shells]
        self.Vown = [self.shells[x].nuclear(self.Rn[x], self.Zn[x]) for x in range(self.nf)]
        self.h = [self.T[x] + self.Vown[x] for x in range(self.nf)]
        self.X = [canonical_orthogonaliser(S) for S in self.S]
        self.Q = [s.schwarz() for s in self.shells]
        self.E_nn_intra = [nuclear_repulsion(self.Zn[x], self.Rn[x]) for x in range(self.nf)]
        self.eri_intra = [I.eri_block(s, s, Q, Q, schwarz) if schwarz > 0 else I.eri_block(s, s)
                          for s, Q in zip(self.shells, self.Q)]
        self.pairs = self.neighbour_pairs(cutoff_A)
        # far field: fragment pairs beyond the cutoff interact through the multipoles (charge, dipole,
        # second moments) of each fragment's nuclei and electrons about its nuclear-charge centroid
        self.far_field = far_field
        near = set(self.pairs)
        self.far_pairs = [(x, y) for x in range(self.nf) for y in range(x + 1, self.nf)
                          if far_field and (x, y) not in near]
        self.centre = [(self.Zn[x][:, None] * self.Rn[x]).sum(0) / self.Zn[x].sum() for x in range(self.nf)]
        if far_field:
            self.M = [self.shells[x].moments(self.centre[x]) for x in range(self.nf)]
            self.Mnuc = []
            for x in range(self.nf):
                r = self.Rn[x] - self.centre[x]
                z = self.Zn[x]
                self.Mnuc.append(np.array([z.sum(), *(z @ r),
                                           z @ (r[:, 0] * r[:, 0]), z @ (r[:, 0] * r[:, 1]), z @ (r[:, 0] * r[:, 2]),
                                           z @ (r[:, 1] * r[:, 1]), z @ (r[:, 1] * r[:, 2]), z @ (r[:, 2] * r[:, 2])]))
        self.nbr = [[] for _ in range(self.nf)]
        for x, y in self.pairs:
            self.nbr[x].append(y)
            self.nbr[y].append(x)
        # V^y on x for every neighbour y (directed), and the inter-fragment ERI block per pair
        self.V = {}
        self.eri = {}
        self.E_nn = {}
        if inter:
            for x, y in self.pairs:
                self.V[(x, y)] = self.shells[x].nuclear(self.Rn[y], self.Zn[y])
                self.V[(y, x)] = self.shells[y].nuclear(self.Rn[x], self.Zn[x])
                self.E_nn[(x, y)] = nuclear_repulsion(self.Zn[x], self.Rn[x], self.Zn[y], self.Rn[y])
                if schwarz > 0:
                    self.eri[(x, y)] = I.eri_block(self.shells[x], self.shells[y], self.Q[x], self.Q[y], schwarz)
                else:
                    self.eri[(x, y)] = I.eri_block(self.shells[x], self.shells[y])

    def neighbour_pairs(self, cutoff_A):
        pairs = []
        xyz = self.system.xyz
        for x in range(self.nf):
            for y in range(x + 1, self.nf):
                if cutoff_A is None:
                    pairs.append((x, y))
                    continue
                d = np.linalg.norm(xyz[self.atoms[x]][:, None, :] - xyz[self.atoms[y]][None, :, :], axis=-1)
                if d.min() < cutoff_A:
                    pairs.append((x, y))
        return pairs

    def shell_quartets(self) -> int:
        """Inter-fragment shell quartets (a<=b in x, c<=d in y, x<y) surviving screening."""
        tau = self.schwarz_tau
        return sum(I.count_quartets(self.shells[x], self.shells[y], self.Q[x], self.Q[y], tau)
                   for x, y in self.pairs)

    # ------------------------------------------------------------------------------------ Fock

    def G(self, x: int, D: np.ndarray) -> np.ndarray:
        """(2J - K) in AO form: G[D] = J[D] - K[D]/2 over the fragment's own AOs."""
        e = self.eri_intra[x]
        return coulomb(e, D) - 0.5 * exchange(e, D)

    def omega(self, Ds) -> list:
        """omega_x = sum_{y in N(x)} (V^y + J[D^y]) for every fragment x (plus the far-field
        multipole terms of the fragments beyond the cutoff when far_field is set)."""
        om = [np.zeros((n, n)) for n in self.n_ao]
        if self.far_field:
            om_far, _ = self.far_terms(Ds)
            om = [o.copy() for o in om_far]
        for x, y in self.pairs:
            e = self.eri[(x, y)]
            nx, ny = self.n_ao[x], self.n_ao[y]
            M = e.reshape(nx * nx, ny * ny)
            om[x] += self.V[(x, y)] + (M @ Ds[y].ravel()).reshape(nx, nx)
            om[y] += self.V[(y, x)] + (M.T @ Ds[x].ravel()).reshape(ny, ny)
        return om

    # ------------------------------------------------------------------------------------ far field

    def multipoles(self, x: int, D: np.ndarray):
        """(q, mu[3], M2[3x3]) of fragment x's nuclei and electrons about its centroid."""
        m = self.Mnuc[x] - np.einsum("kmn,mn->k", self.M[x], D)
        M2 = np.array([[m[4], m[5], m[6]], [m[5], m[7], m[8]], [m[6], m[8], m[9]]])
        return m[0], m[1:4], M2

    @staticmethod
    def interaction_tensors(R):
        """Cartesian derivatives of 1/|R| up to fourth order: T0, T1[a], T2[a,b], T3[a,b,c], T4[a,b,c,d]."""
        r2 = float(R @ R)
        r = math.sqrt(r2)
        d = np.eye(3)
        T0 = 1.0 / r
        T1 = -R / r ** 3
        T2 = (3.0 * np.einsum("a,b->ab", R, R) - r2 * d) / r ** 5
        T3 = (-15.0 * np.einsum("a,b,c->abc", R, R, R) / r ** 7
              + 3.0 * (np.einsum("a,bc->abc", R, d) + np.einsum("b,ac->abc", R, d) + np.einsum("c,ab->abc", R, d))
              / r ** 5)
        RR = np.einsum("a,b->ab", R, R)
        T4 = (105.0 * np.einsum("ab,cd->abcd", RR, RR) / r ** 9
              - 15.0 * (np.einsum("ab,cd->abcd", RR, d) + np.einsum("ac,bd->abcd", RR, d)
                        + np.einsum("ad,bc->abcd", RR, d) + np.einsum("bc,ad->abcd", RR, d)
                        + np.einsum("bd,ac->abcd", RR, d) + np.einsum("cd,ab->abcd", RR, d)) / r ** 7
              + 3.0 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d)) / r ** 5)
        return T0, T1, T2, T3, T4

    def far_potential(self, x: int, y: int, Dy: np.ndarray):
        """(phi, grad phi[3], hess phi[3x3]) at x's centroid of y's multipole expansion:
        phi(r) = q T - mu_a T_a + (1/2) M2_ab T_ab at R = r - c_y (derivatives of 1/|R|)."""
        q, mu, M2 = self.multipoles(y, Dy)
        _, T1, T2, T3, T4 = self.interaction_tensors(self.centre[x] - self.centre[y])
        T0 = 1.0 / np.linalg.norm(self.centre[x] - self.centre[y])
        phi = q * T0 - mu @ T1 + 0.5 * np.einsum("ab,ab->", M2, T2)
        g = q * T1 - np.einsum("a,ac->c", mu, T2) + 0.5 * np.einsum("ab,abc->c", M2, T3)
        H = q * T2 - np.einsum("a,acd->cd", mu, T3) + 0.5 * np.einsum("ab,abcd->cd", M2, T4)
        return phi, g, H

    def far_terms(self, Ds):
        """(omega_far per fragment, E_far per far pair): the Taylor expansion of y's potential about
        x's centroid to second order against x's moments,
        E_xy = q_x phi + mu_x . grad phi + (1/2) M2_x : hess phi,
        and its density derivative for x, -(phi S + grad phi . <r> + (1/2) hess phi : <r r>)."""
        om = [np.zeros((n, n)) for n in self.n_ao]
        E = {}
        for x, y in self.far_pairs:
            for a, b in ((x, y), (y, x)):
                phi, g, H = self.far_potential(a, b, Ds[b])
                M = self.M[a]
                H6 = np.array([H[0, 0], H[0, 1], H[0, 2], H[1, 1], H[1, 2], H[2, 2]])
                w6 = np.array([1.0, 2.0, 2.0, 1.0, 2.0, 1.0])  # off-diagonal second moments appear twice
                om[a] -= phi * M[0] + np.einsum("c,cmn->mn", g, M[1:4]) + 0.5 * np.einsum("k,kmn->mn", w6 * H6, M[4:10])
                if a == x:
                    q, mu, M2 = self.multipoles(x, Ds[x])
                    E[(x, y)] = q * phi + mu @ g + 0.5 * np.einsum("cd,cd->", M2, H)
        return om, E

    def fock(self, Ds) -> list:
        """F^x = h^x + G[D^x] + omega_x for every fragment."""
        om = self.omega(Ds)
        return [self.h[x] + self.G(x, Ds[x]) + om[x] for x in range(self.nf)]

    # ------------------------------------------------------------------------------------ RHF

    def rhf(self, x: int, omega: np.ndarray, D0=None, max_iter: int = 200, diis_size: int = 8,
            e_tol: float = 1e-11, comm_tol: float = 1e-9, shift_after: int = 50, level_shift: float = 0.2):
        """Fragment RHF in a frozen field omega: F = h + omega + G[D], F C = S C eps.

        Canonical orthogonalisation, aufbau occupation of the lowest n_occ orbitals, DIIS (Pulay)
        on the commutator e = F D S - S D F.  Start: D0, else the core guess (F = h + omega).
        A fragment not converged after shift_after iterations restarts from its start density (or
        the core guess) with a fresh DIIS history and its empty orbitals raised by level_shift
        (F' + level_shift (1 - P') in the orthonormal basis, P' the occupied projector of the
        current density): the same self-consistent solutions, a damped path to them.
        Returns (D, F, E_scf, iterations, converged).
        """
        S, X, h = self.S[x], self.X[x], self.h[x]
        nocc = self.n_occ[x]
        hw = h + omega

        def diag(F, D_prev=None, shift=0.0):
            Fo = X.T @ F @ X
            if shift and D_prev is not None:
                Po = X.T @ S @ D_prev @ S @ X / 2.0
                Fo = Fo + shift * (np.eye(Fo.shape[0]) - Po)
            eps, Cp = np.linalg.eigh(Fo)
            C = X @ Cp
            return density_from_orbitals(C[:, :nocc])

        D = diag(hw) if D0 is None else D0
        D_start = D
        Fs, es = [], []
        E_old = None
        shift = 0.0
        for it in range(1, max_iter + 1):
            if shift_after and it == shift_after + 1:
                D, Fs, es, shift = D_start, [], [], level_shift
            F = hw + self.G(x, D)
            E = 0.5 * np.sum(D * (hw + F)) + self.E_nn_intra[x]
            err = F @ D @ S - S @ D @ F
            derr = np.abs(err).max()
            if E_old is not None and abs(E - E_old) < e_tol and derr < comm_tol:
                return D, F, E, it, True
            E_old = E
            Fs.append(F)
            es.append(X.T @ err @ X)
            if len(Fs) > diis_size:
                Fs.pop(0)
                es.pop(0)
            Fx = F
            m = len(Fs)
            if m >= 2:
                B = -np.ones((m + 1, m + 1))
                B[m, m] = 0.0
                for i in range(m):
                    for j in range(m):
                        B[i, j] = np.sum(es[i] * es[j])
                rhs = np.zeros(m + 1)
                rhs[m] = -1.0
                try:
                    c = np.linalg.solve(B, rhs)[:m]
                    Fx = sum(ci * Fi for ci, Fi in zip(c, Fs))
                except np.linalg.LinAlgError:
                    Fx = F
            D = diag(Fx, D, shift)
        return D, F, E, max_iter, False

    # ------------------------------------------------------------------------------------ E_M2

    def e_m2(self, x: int, F: np.ndarray) -> float:
        """Monomer second-order energy of fragment x (Eq. EM2 with the first-order doubles of Eq.
        monDoubles): with the fragment's canonical orbitals (F C = S C eps, canonical
        orthogonalisation, aufbau) the zeroth-order effective Hamiltonian is the diagonal Fock
        operator and the doubles driver is the fragment's own two-electron interaction (the
        environment field is one-body), so that

            E_M2^x = sum_{ij occ, ab virt} (ia|jb) [2 (ia|jb) - (ib|ja)] / (eps_i + eps_j - eps_a - eps_b).
        """
        X = self.X[x]
        nocc = self.n_occ[x]
        eps, Cp = np.linalg.eigh(X.T @ F @ X)
        C = X @ Cp
        Co, Cv = C[:, :nocc], C[:, nocc:]
        eo, ev = eps[:nocc], eps[nocc:]
        eri = I.eri_block(self.shells[x], self.shells[x])  # unscreened (mu nu|lambda sigma)
        ovov = np.einsum("mi,na,mnls,lj,sb->iajb", Co, Cv, eri, Co, Cv, optimize=True)
        den = eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] - ev[None, None, None, :]
        return float(np.sum(ovov * (2.0 * ovov - ovov.transpose(0, 3, 2, 1)) / den))

    def canonical_orbitals(self, x: int, F: np.ndarray):
        """(C, eps): canonical orbitals of F^x (F C = S C eps via the canonical orthogonaliser)."""
        X = self.X[x]
        eps, Cp = np.linalg.eigh(X.T @ F @ X)
        return X @ Cp, eps

    def e_d2(self, x: int, y: int, Fx: np.ndarray, Fy: np.ndarray) -> float:
        """Dimer second-order energy of the pair (x, y) (Eq. ED2 with the first-order dimer doubles of
        Eq. dimDoubles): one excitation on each fragment, direct interaction only (the product
        ansatz has no inter-fragment exchange), four spin cases:

            E_D2^{xy} = 4 sum_{i,a in x; j,b in y} (ia|jb)^2 / (eps_i + eps_j - eps_a - eps_b).
        """
        Cx, ex = self.canonical_orbitals(x, Fx)
        Cy, ey = self.canonical_orbitals(y, Fy)
        ox, oy = self.n_occ[x], self.n_occ[y]
        eri = I.eri_block(self.shells[x], self.shells[y])  # unscreened (mu nu|lambda sigma), mu nu in x
        ovov = np.einsum("mi,na,mnls,lj,sb->iajb", Cx[:, :ox], Cx[:, ox:], eri, Cy[:, :oy], Cy[:, oy:],
                         optimize=True)
        den = (ex[:ox, None, None, None] - ex[None, ox:, None, None] + ey[None, None, :oy, None]
               - ey[None, None, None, oy:])
        return float(4.0 * np.sum(ovov * ovov / den))

    # ------------------------------------------------------------------------------------ energies

    def energies(self, Ds) -> dict:
        """Reference energies of the Hartree product.

        E_x^int = tr[D^x (2 h^x + G[D^x])]/2 + sum_{A<B in x} Z_A Z_B / R_AB
        E_xy    = tr[D^x V^y] + tr[D^y V^x] + tr[D^x J[D^y]] + sum_{A in x, B in y} Z_A Z_B / R_AB
        E_tot   = sum_x E_x^int + sum_{pairs x<y} E_xy
        E_x     = E_x^int + (1/2) sum_{y in N(x)} E_xy      (so that sum_x E_x = E_tot)
        E_x^scf = E_x^int + tr[D^x omega_x]
        """
        nf = self.nf
        E_int = np.array([0.5 * np.sum(Ds[x] * (2 * self.h[x] + self.G(x, Ds[x]))) + self.E_nn_intra[x]
                          for x in range(nf)])
        E_pair = {}
        for x, y in self.pairs:
            nx, ny = self.n_ao[x], self.n_ao[y]
            Jxy = coulomb(self.eri[(x, y)], Ds[y])
            E_pair[(x, y)] = (np.sum(Ds[x] * self.V[(x, y)]) + np.sum(Ds[y] * self.V[(y, x)]) +
                              np.sum(Ds[x] * Jxy) + self.E_nn[(x, y)])
        if self.far_field:
            _, E_far = self.far_terms(Ds)
            E_pair.update(E_far)
        E_x = E_int.copy()
        for (x, y), e in E_pair.items():
            E_x[x] += 0.5 * e
            E_x[y] += 0.5 * e
        om = self.omega(Ds)
        E_scf = np.array([E_int[x] + np.sum(Ds[x] * om[x]) for x in range(nf)])
        E_tot = float(E_int.sum() + sum(E_pair.values()))
        return dict(E_int=E_int, E_pair=E_pair, E_x=E_x, E_tot=E_tot, E_scf=E_scf)

    # ------------------------------------------------------------------------------------ FEF loop

    def isolated(self, **kw):
        """Isolated-fragment RHF densities (omega = 0): the superposition start."""
        out = []
        for x in range(self.nf):
            D, F, E, it, ok = self.rhf(x, np.zeros_like(self.h[x]), **kw)
            if not ok:
                raise RuntimeError(f"isolated RHF of fragment {x} did not converge")
            out.append(D)
        return out

    def solve(self, D0=None, e_tol: float = 1e-8, max_macro: int = 100, **rhf_kw):
        """FEF self-consistency.

        D^(0): superposition of isolated-fragment RHF densities (or D0).  Macro-iteration k builds
        omega^(k) from D^(k-1) of all fragments, then solves every fragment's RHF in its frozen
        omega^(k) to get D^(k).  Stops when |dE_tot| < e_tol and max_x |dE_x| < e_tol.
        Returns dict(D, F, energies, n_macro, converged, history).
        """
        Ds = self.isolated(**rhf_kw) if D0 is None else [d.copy() for d in D0]
        En = self.energies(Ds)
        history = [En["E_tot"]]
        for k in range(1, max_macro + 1):
            om = self.omega(Ds)
            new = []
            for x in range(self.nf):
                D, F, E, it, ok = self.rhf(x, om[x], D0=Ds[x], **rhf_kw)
                if not ok:
                    raise RuntimeError(f"fragment {x} RHF in the field did not converge at macro {k}")
                new.append(D)
            Ds = new
            En_new = self.energies(Ds)
            history.append(En_new["E_tot"])
            dE = abs(En_new["E_tot"] - En["E_tot"])
            dEx = np.abs(En_new["E_x"] - En["E_x"]).max()
            En = En_new
            if dE < e_tol and dEx < e_tol:
                return dict(D=Ds, F=self.fock(Ds), energies=En, n_macro=k, converged=True, history=history)
        return dict(D=Ds, F=self.fock(Ds), energies=En, n_macro=max_macro, converged=False, history=history)
