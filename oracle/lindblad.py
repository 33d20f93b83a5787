"""The AME generator frozen at one point s, in the instantaneous eigenframe.

Test infrastructure only (see the package docstring).

Sec. II, Eqs. ME2-H, ME2-L and Lindblad2, with a diagonal rate matrix
(independent baths, App. F) and the rates absorbed into the operators (Sec. III,
Eq. Aired). In the eigenframe of H_S(s) (columns of V), with
M_alpha = V^T sz_alpha V, the jump operator of qubit alpha and Bohr class c is

    A_{alpha,c} = sum_{(a,b) in c} sqrt(gamma(omega_ab)) M_alpha[a,b] |a><b| ,

omega_ab = E(m(b)) - E(m(a)) (the frequency of the transition b -> a), and the
effective Hamiltonian (Sec. III, Eq. Heff) is

    K = diag(eps) + H_LS - (i/2) sum_{alpha,c} A^dag A ,
    H_LS = sum_{alpha,c} S(omega) L^dag L  (App. E).

Both sums reduce to K[b,b'] = eps_b delta + sum_alpha sum_a f(omega_ab) M[a,b] M[a,b']
for b, b' in the same degenerate manifold (zero otherwise), f = S - (i/2) gamma:
two pairs of one class that share the target level a have sources of equal energy.
"""
from __future__ import annotations

import numpy as np

from . import bath, model


class Frame:
    """Generator data at one grid point."""

    def __init__(self, inst, s: float, terms=None, zdiag=None, wmax=None):
        n = inst.n_qubits
        self.eig = eig = model.eigen_at(inst, s, terms)
        self.N = N = len(eig.evals)
        z = model.sigma_z_diagonals(n) if zdiag is None else zdiag
        V = eig.V
        self.M = np.array([V.T @ (z[al][:, None] * V) for al in range(n)])
        w = eig.omega  # w[a, b]: Bohr frequency of b -> a
        self.gam = bath.gamma(w, inst.eta_g2, inst.omega_c, inst.beta)
        if inst.lamb_shift:
            wmax = wmax if wmax is not None else max(50.0, float(np.max(np.abs(w))))
            self.S = bath.lamb_shift(w, inst.eta_g2, inst.omega_c, inst.beta, wmax=wmax)
        else:
            self.S = np.zeros_like(w)
        self.R = np.sqrt(self.gam)[None, :, :] * self.M  # R[alpha, a, b]
        same = eig.level_manifold[:, None] == eig.level_manifold[None, :]
        self.same = same
        f = self.S - 0.5j * self.gam
        K = np.diag(eig.evals).astype(complex)
        for al in range(n):
            K += ((f * self.M[al]).T @ self.M[al]) * same
        self.K = K
        # Bohr classes as level-pair masks (Eq. Lindblad2).
        self.classes = model.bohr_classes(eig)
        lm = eig.level_manifold
        nm = len(eig.E)
        cid = np.full((nm, nm), -1, dtype=int)
        for ci, (_, pairs) in enumerate(self.classes):
            if len(pairs) == 1:
                cid[pairs[0]] = ci
            else:
                pa = np.array(pairs)
                cid[pa[:, 0], pa[:, 1]] = ci
        self.class_of_pair = cid[lm[:, None], lm[None, :]]  # [a, b] -> class id
        # Sort the level pairs of each class into three evaluation shapes.
        order = np.argsort(self.class_of_pair, axis=None, kind="stable")
        flat = self.class_of_pair.reshape(-1)[order]
        starts = np.flatnonzero(np.r_[True, flat[1:] != flat[:-1]])
        ends = np.r_[starts[1:], len(flat)]
        sizes = ends - starts
        single = starts[sizes == 1]
        self.sing_a, self.sing_b = np.divmod(order[single], N)
        self.diag_classes, self.dense_classes = [], []
        for st, en in zip(starts[sizes > 1], ends[sizes > 1]):
            ia, ib = np.divmod(order[st:en], N)
            if np.all(ia == ib):
                self.diag_classes.append(ia)
            else:
                self.dense_classes.append((ia, ib))
        # Rate of each singleton pair summed over alpha: sum_alpha R[alpha,a,b]^2.
        self.sing_rate = np.sum(self.R[:, self.sing_a, self.sing_b] ** 2, axis=0)

    # ----- the Lindblad generator (matrix-free) -------------------------------
    def apply(self, rho: np.ndarray) -> np.ndarray:
        """L[rho] = -i (K rho - rho K^dag) + sum_{alpha,c} A rho A^dag  (Eq. effdiagonalform)."""
        out = -1j * (self.K @ rho - rho @ self.K.conj().T)
        N = self.N
        if len(self.sing_a):
            pops = np.diagonal(rho)[self.sing_b] * self.sing_rate
            out[np.diag_indices(N)] += np.bincount(self.sing_a, weights=pops.real, minlength=N) \
                + 1j * np.bincount(self.sing_a, weights=pops.imag, minlength=N)
        for ia in self.diag_classes:
            sub = rho[np.ix_(ia, ia)]
            acc = np.zeros_like(sub)
            for al in range(self.R.shape[0]):
                v = self.R[al, ia, ia]
                acc += np.outer(v, v) * sub
            out[np.ix_(ia, ia)] += acc
        for ia, ib in self.dense_classes:
            for al in range(self.R.shape[0]):
                A = np.zeros((N, N))
                A[ia, ib] = self.R[al, ia, ib]
                out += A @ rho @ A.T
        return out

    def norm_bound(self) -> float:
        return 2.0 * np.max(np.sum(np.abs(self.K), axis=1)) + float(np.sum(self.R ** 2))

    def propagate(self, rho: np.ndarray, tau: float) -> np.ndarray:
        """exp(L tau) rho by its Taylor series, on substeps with ||L|| tau_sub <= 1/2."""
        nsub = max(1, int(np.ceil(self.norm_bound() * tau / 0.5)))
        h = tau / nsub
        for _ in range(nsub):
            term = rho
            acc = rho.copy()
            for j in range(1, 80):
                term = self.apply(term) * (h / j)
                acc = acc + term
                if np.max(np.abs(term)) <= 1e-18 * max(1e-300, np.max(np.abs(acc))):
                    break
            rho = acc
        return rho

    # ----- generic-spectrum closed form ---------------------------------------
    @property
    def generic(self) -> bool:
        """Nondegenerate spectrum and every class other than omega = 0 holds one pair."""
        if not self.eig.nondegenerate:
            return False
        return all(len(p) == 1 for _, p in self.classes[1:])

    def propagate_generic(self, rho: np.ndarray, tau: float) -> np.ndarray:
        """exp(L tau) rho when ``generic``: the generator then decouples into a
        rate equation for the populations and independent coherences."""
        from scipy.linalg import expm
        R2 = np.sum(self.R ** 2, axis=0)  # R2[a, b] = sum_alpha gamma M^2
        W = R2.copy()
        np.fill_diagonal(W, 0.0)
        W -= np.diag(W.sum(axis=0))
        d = np.array([np.diag(r) for r in self.R])  # d[alpha, a] = R[alpha, a, a]
        Kd = np.diag(self.K)
        lam = -1j * (Kd[:, None] - Kd.conj()[None, :]) + d.T @ d
        out = np.exp(lam * tau) * rho
        p = expm(W * tau) @ np.real(np.diag(rho))
        np.fill_diagonal(out, p)
        return out

    # ----- dense superoperator (small N; used by the pins) ----------------------
    def superoperator(self) -> np.ndarray:
        """L as an N^2 x N^2 matrix on row-major vec(rho), built entry by entry
        from the four-index form of the jump term."""
        N = self.N
        I = np.eye(N)
        Lsup = -1j * (np.kron(self.K, I) - np.kron(I, self.K.conj()))
        cp = self.class_of_pair
        same_class = cp[:, None, :, None] == cp[None, :, None, :]  # [a, a', b, b']
        T = np.zeros((N, N, N, N))
        for al in range(self.R.shape[0]):
            T += self.R[al][:, None, :, None] * self.R[al][None, :, None, :]
        T = T * same_class
        return Lsup + T.reshape(N * N, N * N)
