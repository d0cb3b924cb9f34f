"""Plain FP64 CPU oracle of the discrete Kohn-Sham model.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py, never by the product library.

Discrete model (paper Sec. 5.1, plane-wave discretisation of Eq. (1.1)/(1.4),
H as the DFTK-style Hamiltonian -1/2 Laplacian + V of Sec. 5.2):
  * cubic cell of edge a, volume Omega = a^3, reciprocal spacing b = 2 pi / a;
  * real-space grid r_j = a j / N, j in {0..N-1}^3, arrays indexed [jx, jy, jz];
  * at k = b * kfrac the basis is {G = b m : 1/2 |k+G|^2 <= Ecut}, m with
    components in [-N/2, N/2), canonical order lexicographic (mx, my, mz), mz fastest;
  * orbital on the grid u(r_j) = Omega^{-1/2} sum_G c_G exp(i G.r_j);
  * density rho = sum_k w_k f sum_i |u_ik|^2, integral (Omega/N^3) sum_j;
  * V_loc(G) = sum_a -4 pi Z_a/(Omega |G|^2) exp(-|G|^2 rc_a^2/4) exp(-i G.R_a), G != 0;
  * V_H(G) = 4 pi rho(G)/|G|^2 (G != 0), V_x = -(3 rho/pi)^{1/3} (Slater exchange);
  * xc = 2 adds LDA correlation: the spin-unpolarised Perdew-Wang 1992 fit of the homogeneous
    electron gas correlation energy per electron, eps_c(r_s), r_s = (3 / (4 pi rho))^{1/3},
    E_c = int rho eps_c, V_c = eps_c - (r_s / 3) d eps_c / d r_s (the paper's experiments use
    DFTK's LDA model, Sec. 5.3; its correlation is this fit; the fitted constants alpha1,
    beta3, beta4: parity unpinned beyond a 1 mHa agreement with the Perdew-Zunger fit);
  * Nyquist planes and G = 0 of every potential are zero;
  * s/p Gaussian projectors beta_al(G) = Omega^{-1/2} F_l(k+G) exp(-i (k+G).R_a)
    with coupling D_al; E_nl = sum_k w_k f sum_i sum_al D_al |<beta_al, c_i>|^2;
  * H is the exact derivative of this discrete energy: DE[W] = 2 f <H Phi, W>
    with the pairing <V, W> = sum_k w_k Re tr(V_k^* W_k) (Eq. (2.4)).

Blocks are numpy arrays of shape (n_k, p): column i is orbital i (Sec. 5.1).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

WORKERS = -1  # scipy.fft threads: all host cores


def _fftn(x, axes=(-3, -2, -1)):
    return sfft.fftn(x, axes=axes, workers=WORKERS)


def _ifftn(x, axes=(-3, -2, -1)):
    return sfft.ifftn(x, axes=axes, workers=WORKERS)


def sphere_threshold(ecut: float, b: float) -> float:
    """The basis test 1/2 |k+G|^2 <= Ecut in units of b: |kfrac + m|^2 <= 2 Ecut / b^2."""
    return (2.0 * ecut) / (b * b)


def sphere_basis(N: int, kfrac, ecut: float, b: float):
    """Integer triples m of the plane-wave basis at one k (Sec. 5.1), canonical order.

    The floating-point decision is taken as s = (mx+kx)^2 + (my+ky)^2 + (mz+kz)^2
    (each square rounded, summed left to right, no fused multiply-add) compared
    with sphere_threshold(ecut, b)."""
    m1 = np.arange(-(N // 2), N - N // 2, dtype=np.int64)
    mx, my, mz = np.meshgrid(m1, m1, m1, indexing="ij")
    M = np.stack([mx.ravel(), my.ravel(), mz.ravel()], axis=1)
    q = M.astype(np.float64) + np.asarray(kfrac, np.float64)[None, :]
    s = (q[:, 0] * q[:, 0] + q[:, 1] * q[:, 1]) + q[:, 2] * q[:, 2]
    return M[s <= sphere_threshold(ecut, b)]


def frequencies(N: int):
    """Signed integer frequency of each FFT index, Nyquist (-N/2) flagged."""
    f = np.fft.fftfreq(N, d=1.0 / N).astype(np.int64)
    nyq = (f == -(N // 2)) if N % 2 == 0 else np.zeros(N, bool)
    return f, nyq


# Perdew-Wang 1992 parameters of the spin-unpolarised correlation energy (Table I, zeta = 0)
PW92 = dict(A=0.031091, alpha1=0.21370, beta1=7.5957, beta2=3.5876, beta3=1.6382, beta4=0.49294)


class Model:
    """One synthetic crystal (config dict from the synth module) on one FFT grid."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.a = float(cfg["a"])
        self.N = int(cfg["N"])
        self.omega = self.a ** 3
        self.b = 2.0 * math.pi / self.a
        self.ecut = float(cfg["ecut"])
        self.kfrac = np.asarray(cfg["kfrac"], np.float64).reshape(-1, 3)
        self.kw = np.asarray(cfg["kweight"], np.float64)
        self.K = len(self.kfrac)
        self.p = int(cfg["nbands"])
        self.occ = float(cfg["occ"])
        self.pos = np.asarray(cfg["pos"], np.float64).reshape(-1, 3)
        self.Z = np.asarray(cfg["Z"], np.float64)
        self.rc = np.asarray(cfg["rc"], np.float64)
        self.nproj_per_atom = int(cfg["nproj_per_atom"])
        self.width = float(cfg["proj_width"])
        self.D = np.asarray(cfg["D"], np.float64).reshape(-1, 2)
        self.hartree = int(cfg["hartree"])
        self.xc = int(cfg["xc"])
        N = self.N
        self.basis = [sphere_basis(N, kf, self.ecut, self.b) for kf in self.kfrac]
        self.nk = [len(m) for m in self.basis]
        # flat grid index of each basis vector (FFT index m mod N)
        self.gidx = [((m[:, 0] % N) * N + (m[:, 1] % N)) * N + (m[:, 2] % N) for m in self.basis]
        # 1/2 |k+G|^2 per basis vector
        self.kin = [0.5 * (self.b ** 2) * ((m + kf[None, :]) ** 2).sum(1)
                    for m, kf in zip(self.basis, self.kfrac)]
        f, nyq = frequencies(N)
        FX, FY, FZ = np.meshgrid(f, f, f, indexing="ij")
        self.G2 = (self.b ** 2) * (FX ** 2 + FY ** 2 + FZ ** 2).astype(np.float64)
        self.gmask = ~(nyq[:, None, None] | nyq[None, :, None] | nyq[None, None, :])
        self.gmask &= self.G2 > 0
        self.Gvec = [self.b * FX, self.b * FY, self.b * FZ]
        self.vloc = self._local_potential()
        self.proj = [self._projectors(k) for k in range(self.K)]
        self.Dvec = self._coupling_vector()

    # ------------------------------------------------------------------ potentials
    def _local_potential(self):
        """V_loc on the grid: sum over G of the Gaussian-screened ionic term (Sec. 1,
        Eq. (1.1) ionic part; the synthetic form factor of the workloads)."""
        N = self.N
        vg = np.zeros((N, N, N), np.complex128)
        G2 = self.G2
        m = self.gmask
        for R, Z, rc in zip(self.pos, self.Z, self.rc):
            phase = np.exp(-1j * (self.Gvec[0] * R[0] + self.Gvec[1] * R[1] + self.Gvec[2] * R[2]))
            term = np.zeros_like(vg)
            term[m] = -4.0 * math.pi * Z / (self.omega * G2[m]) * np.exp(-G2[m] * rc * rc / 4.0) * phase[m]
            vg += term
        return (N ** 3 * _ifftn(vg)).real

    def hartree_potential(self, rho):
        """V_H(G) = 4 pi rho(G) / |G|^2 with rho(G) = N^-3 sum_j rho_j e^{-iG.r_j}."""
        N = self.N
        rg = _fftn(rho.astype(np.complex128)) / N ** 3
        vg = np.zeros_like(rg)
        vg[self.gmask] = 4.0 * math.pi * rg[self.gmask] / self.G2[self.gmask]
        return (N ** 3 * _ifftn(vg)).real

    @staticmethod
    def exchange_potential(rho):
        """Slater exchange potential -(3 rho / pi)^{1/3}, derivative of -3/4 (3/pi)^{1/3} rho^{4/3}."""
        return -np.cbrt(3.0 * np.maximum(rho, 0.0) / math.pi)

    @staticmethod
    def exchange_energy_density(rho):
        return -0.75 * np.cbrt(3.0 / math.pi) * np.maximum(rho, 0.0) ** (4.0 / 3.0)

    @staticmethod
    def correlation(rho):
        """Perdew-Wang 1992 LDA correlation (spin-unpolarised; Phys. Rev. B 45, 13244, Eq. (10)
        with the zeta = 0 column of its Table I):
            eps_c(r_s) = -2 A (1 + alpha1 r_s) ln(1 + 1 / (2 A (beta1 r_s^1/2 + beta2 r_s
                                                          + beta3 r_s^3/2 + beta4 r_s^2))).
        Returns (rho eps_c, V_c) with V_c = d(rho eps_c)/d rho = eps_c - (r_s/3) eps_c'(r_s);
        both are 0 where rho <= 0."""
        A, a1 = PW92["A"], PW92["alpha1"]
        b1, b2, b3, b4 = PW92["beta1"], PW92["beta2"], PW92["beta3"], PW92["beta4"]
        rho = np.asarray(rho, np.float64)
        pos = rho > 0.0
        rs = np.where(pos, np.cbrt(3.0 / (4.0 * math.pi * np.where(pos, rho, 1.0))), 1.0)
        sq = np.sqrt(rs)
        q0 = -2.0 * A * (1.0 + a1 * rs)
        q1 = 2.0 * A * (b1 * sq + b2 * rs + b3 * rs * sq + b4 * rs * rs)
        dq1 = A * (b1 / sq + 2.0 * b2 + 3.0 * b3 * sq + 4.0 * b4 * rs)
        lg = np.log1p(1.0 / q1)
        eps = q0 * lg
        deps = -2.0 * A * a1 * lg - q0 * dq1 / (q1 * q1 + q1)
        vc = eps - rs / 3.0 * deps
        return np.where(pos, rho * eps, 0.0), np.where(pos, vc, 0.0)

    def potentials(self, rho):
        """Total potential V_tot = V_loc + V_H + V_xc and its Hartree/exchange-correlation parts."""
        vh = self.hartree_potential(rho) if self.hartree else np.zeros_like(rho)
        vx = self.exchange_potential(rho) if self.xc else np.zeros_like(rho)
        if self.xc == 2:
            vx = vx + self.correlation(rho)[1]
        return self.vloc + vh + vx, vh, vx

    # ------------------------------------------------------------------ projectors
    def form_factors(self, q):
        """F_s and F_p,alpha of the L2-normalised Gaussian s/p projectors (width w):
        s(r) = (pi w^2)^{-3/4} e^{-r^2/2w^2},  p_a(r) = (2/w^2)^{1/2} x_a s(r);
        F(q) = int f(r) e^{-i q.r} dr.  q is (n, 3); returns (n, 4) complex."""
        w = self.width
        q2 = (q ** 2).sum(1)
        g = np.exp(-q2 * w * w / 2.0)
        Fs = 2.0 ** 1.5 * math.pi ** 0.75 * w ** 1.5 * g
        cp = -1j * w * w * (2.0 * math.pi * w * w) ** 1.5 * math.sqrt(2.0 / (w * w)) * (math.pi * w * w) ** -0.75
        out = np.empty((len(q), 4), np.complex128)
        out[:, 0] = Fs
        for al in range(3):
            out[:, 1 + al] = cp * q[:, al] * g
        return out

    def _projectors(self, k):
        """B_k (n_k x nproj): beta_al(G) = Omega^{-1/2} F_l(k+G) e^{-i (k+G).R_a},
        projectors ordered atom-major, within an atom s, px, py, pz (first nproj_per_atom)."""
        npa = self.nproj_per_atom
        if npa == 0:
            return np.zeros((self.nk[k], 0), np.complex128)
        q = self.b * (self.basis[k] + self.kfrac[k][None, :])
        F = self.form_factors(q)
        cols = []
        for R in self.pos:
            ph = np.exp(-1j * (q @ R)) / math.sqrt(self.omega)
            for l in range(npa):
                cols.append(F[:, l] * ph)
        return np.stack(cols, axis=1)

    def _coupling_vector(self):
        npa = self.nproj_per_atom
        d = []
        for Da in self.D:
            for l in range(npa):
                d.append(Da[0] if l == 0 else Da[1])
        return np.asarray(d, np.float64)

    # ------------------------------------------------------------------ grid maps
    def to_grid(self, k, C):
        """u(r_j) for each column of C: Omega^{-1/2} sum_G c_G e^{iG.r_j}; shape (p, N, N, N)."""
        N = self.N
        p = C.shape[1]
        g = np.zeros((p, N ** 3), np.complex128)
        g[:, self.gidx[k]] = C.T
        g = g.reshape(p, N, N, N)
        return (N ** 3 / math.sqrt(self.omega)) * _ifftn(g)

    def density(self, Phi):
        """rho(r_j) = sum_k w_k f sum_i |u_ik(r_j)|^2."""
        N = self.N
        rho = np.zeros((N, N, N))
        for k in range(self.K):
            u = self.to_grid(k, Phi[k])
            rho += self.kw[k] * self.occ * (np.abs(u) ** 2).sum(0)
        return rho

    def integrate(self, g):
        return self.omega / self.N ** 3 * g.sum()

    # ------------------------------------------------------------------ H and E
    def apply_H(self, k, C, vtot):
        """H_k C: kinetic 1/2|k+G|^2 c_G, plus local part restricted to the sphere,
        (1/N^3) FFT(V_tot * IFFT_unnormalised(c)) = fftn(V_tot * ifftn(c)), plus nonlocal B D B^* C."""
        N = self.N
        p = C.shape[1]
        out = self.kin[k][:, None] * C
        g = np.zeros((p, N ** 3), np.complex128)
        g[:, self.gidx[k]] = C.T
        g = g.reshape(p, N, N, N)
        w = _fftn(vtot[None] * _ifftn(g)).reshape(p, N ** 3)
        out = out + w[:, self.gidx[k]].T
        B = self.proj[k]
        if B.shape[1]:
            out = out + B @ (self.Dvec[:, None] * (B.conj().T @ C))
        return out

    def energy_terms(self, Phi, rho=None):
        """Kinetic, local, Hartree, exchange and nonlocal energies (Eq. (1.1) discretised)."""
        if rho is None:
            rho = self.density(Phi)
        ekin = 0.0
        enl = 0.0
        for k in range(self.K):
            C = Phi[k]
            ekin += self.kw[k] * self.occ * float((self.kin[k][:, None] * np.abs(C) ** 2).sum())
            B = self.proj[k]
            if B.shape[1]:
                P = B.conj().T @ C
                enl += self.kw[k] * self.occ * float((self.Dvec[:, None] * np.abs(P) ** 2).sum())
        eloc = self.integrate(self.vloc * rho)
        eh = 0.5 * self.integrate(self.hartree_potential(rho) * rho) if self.hartree else 0.0
        ex = self.integrate(self.exchange_energy_density(rho)) if self.xc else 0.0
        if self.xc == 2:
            ex += self.integrate(self.correlation(rho)[0])
        return dict(kin=ekin, loc=float(eloc), hartree=float(eh), xc=float(ex), nl=enl)

    def energy(self, Phi, rho=None):
        return float(sum(self.energy_terms(Phi, rho).values()))

    # ------------------------------------------------------------------ dense H
    def dense_H(self, k, vtot):
        """Explicit n_k x n_k matrix: 1/2|k+G|^2 delta + V(G - G') + B D B^*, with
        V(G) = N^-3 sum_j V_j e^{-iG.r_j} read at the grid frequency (m - m') mod N."""
        N = self.N
        vg = _fftn(vtot.astype(np.complex128)) / N ** 3
        m = self.basis[k]
        d = (m[:, None, :] - m[None, :, :]) % N
        H = vg[d[..., 0], d[..., 1], d[..., 2]]
        H = H + np.diag(self.kin[k])
        B = self.proj[k]
        if B.shape[1]:
            H = H + B @ (self.Dvec[:, None] * B.conj().T)
        return H


def pairing(model: Model, V, W) -> float:
    """<V, W> = sum_k w_k Re tr(V_k^* W_k): the real Frobenius pairing (Sec. 2.1, Sec. 5.1)
    summed over the product manifold (Eq. (5.1)) with k-point weights."""
    return float(sum(model.kw[k] * np.vdot(V[k], W[k]).real for k in range(model.K)))


def residual_norm(R) -> float:
    """||R||_F over all k-points (unweighted), the convergence measure of Sec. 5.3."""
    return math.sqrt(sum(float(np.vdot(r, r).real) for r in R))
