"""Fermion matrix M[phi] and M^dagger[phi] (oracle; test infrastructure only).

Two forms are restated here.

Exponential-hopping form (the form the GPU library computes).  With the
transfer matrix E = exp(delta*kappa*h) on every time slice, the phases
D_t = diag(exp(i phi_{x,t})) of the auxiliary field (Eq. (2.2) attaches
exp(i delta phi_{x,t}) to the time hop; phi here already carries the delta) and
the antiperiodic time boundary of fermions:

    (M psi)_t      = psi_t - s_t     * E D_{t-1} psi_{t-1}
    (M^dag psi)_t  = psi_t - s_{t+1} * D_t^* E psi_{t+1}
    s_0 = -1, s_t = +1 (t != 0), time indices mod Nt

so det M = det(1 + E D_{Nt-1} ... E D_0) and at phi = 0, det M =
prod_lambda (1 + exp(beta kappa lambda)) over the eigenvalues lambda of h.

Mixed-differencing form printed as Eq. (2.2) (Brower-Rebbi-Schaich): on A
sites a forward time difference with exp(+i phi_{x,t}) on the diagonal, on B
sites a backward difference with exp(-i phi_{x,t}) on the sub-diagonal, and
-delta*kappa hopping within the slice.  Antiperiodic wrap: psi_{x,Nt} =
-psi_{x,0} and psi_{x,-1} = -psi_{x,Nt-1}.
"""
import numpy as np

from . import lattice


# ---------------------------------------------------------------------------
# transfer matrix
# ---------------------------------------------------------------------------
def transfer_matrix(h, delta_kappa, delta_mu=0.0):
    """E = exp(delta*kappa*h - delta*mu) through the eigendecomposition of
    the real symmetric h: E = Q diag(exp(delta*kappa*w - delta*mu)) Q^T.
    The chemical potential mu (the sign-problem setting of §3,
    p ~ det(M[phi,mu] M[phi,-mu]^dag)) is the one of the particle-hole
    Hamiltonian of §1, whose term + mu sum_x rho_x with
    rho_x = p^dag p - h^dag h gives the particles the Boltzmann factor
    e^{-delta mu} per slice (M[phi,mu]) and the holes e^{+delta mu}
    (M[phi,-mu]); delta_mu = 0 is half filling."""
    w, Q = np.linalg.eigh(h)
    return (Q * np.exp(delta_kappa * w - delta_mu)) @ Q.T


def time_signs(Nt):
    """s_t of the antiperiodic boundary: s_0 = -1, others +1."""
    s = np.ones(Nt, dtype=np.float64)
    s[0] = -1.0
    return s


# ---------------------------------------------------------------------------
# exponential form, matrix free.  phi: (Nt, V) real, psi: (Nt, V) complex
# ---------------------------------------------------------------------------
def apply_M(E, phi, psi):
    """(M psi)_t = psi_t - s_t E (e^{i phi_{t-1}} * psi_{t-1})."""
    Nt = phi.shape[0]
    u = np.exp(1j * phi) * psi                 # D_t psi_t on every slice
    w = u @ E.T                                # w_t = E u_t  (row t of w)
    w_prev = np.roll(w, 1, axis=0)             # w_prev[t] = w[t-1 mod Nt]
    return psi - time_signs(Nt)[:, None] * w_prev


def apply_Mdag(E, phi, psi):
    """(M^dag psi)_t = psi_t - s_{t+1} e^{-i phi_t} * (E psi_{t+1})."""
    Nt = phi.shape[0]
    w = psi @ E.T                              # w_t = E psi_t
    w_next = np.roll(w, -1, axis=0)            # w_next[t] = w[t+1 mod Nt]
    s_next = np.roll(time_signs(Nt), -1)       # s_{t+1}
    return psi - s_next[:, None] * np.exp(-1j * phi) * w_next


def apply_MMdag(E, phi, psi):
    return apply_M(E, phi, apply_Mdag(E, phi, psi))


# ---------------------------------------------------------------------------
# exponential form, dense (tiny lattices only; pure-Python block loop)
# ---------------------------------------------------------------------------
def dense_M(E, phi):
    """N x N matrix of the exponential form, N = Nt*V, index t*V + x.
    Built slice block by slice block straight from the definition."""
    Nt, V = phi.shape
    N = Nt * V
    M = np.eye(N, dtype=np.complex128)
    s = time_signs(Nt)
    for t in range(Nt):
        tp = (t - 1) % Nt
        D = np.exp(1j * phi[tp])
        block = E * D[None, :]                 # E @ diag(D)
        M[t * V:(t + 1) * V, tp * V:(tp + 1) * V] -= s[t] * block
    return M


def reduced_matrix(E, phi):
    """1 + E D_{Nt-1} E D_{Nt-2} ... E D_0  (V x V); det of it equals det M."""
    Nt, V = phi.shape
    P = np.eye(V, dtype=np.complex128)
    for t in range(Nt):
        P = (E * np.exp(1j * phi[t])[None, :]) @ P
    return np.eye(V) + P


# ---------------------------------------------------------------------------
# printed mixed-differencing form, Eq. (2.2)
# ---------------------------------------------------------------------------
def dense_M_brs(L, phi, delta, kappa):
    """Dense N x N matrix of Eq. (2.2) with phi already multiplied by delta.
    Loops over every (row, column) block entry the equation defines."""
    Nt, V = phi.shape
    N = Nt * V
    sub = lattice.sublattice(L)
    h = lattice.hopping_matrix(L)
    M = np.zeros((N, N), dtype=np.complex128)

    def col(x, t):
        # antiperiodic wrap: returns (column index, sign)
        if t == Nt:
            return x, -1.0
        if t == -1:
            return (Nt - 1) * V + x, -1.0
        return t * V + x, 1.0

    for t in range(Nt):
        for x in range(V):
            row = t * V + x
            if sub[x] == 0:        # A: delta_{t+1,t'} - delta_{t,t'} e^{+i phi_{x,t}}
                c, sg = col(x, t + 1)
                M[row, c] += sg
                M[row, t * V + x] -= np.exp(1j * phi[t, x])
            else:                  # B: delta_{t,t'} - delta_{t-1,t'} e^{-i phi_{x,t}}
                M[row, t * V + x] += 1.0
                c, sg = col(x, t - 1)
                M[row, c] -= sg * np.exp(-1j * phi[t, x])
            for y in range(V):     # AB / BA: -delta kappa delta_<x,y> delta_{t,t'}
                if h[x, y] != 0.0:
                    M[row, t * V + y] -= delta * kappa * h[x, y]
    return M


def apply_M_brs(L, phi, psi, delta, kappa):
    """Matrix-free form of Eq. (2.2) (same conventions as dense_M_brs)."""
    Nt, V = phi.shape
    sub = lattice.sublattice(L)
    h = lattice.hopping_matrix(L)
    isA = (sub == 0)[None, :]
    fwd = np.roll(psi, -1, axis=0)             # psi_{t+1}
    fwd[Nt - 1] *= -1.0
    bwd = np.roll(psi, 1, axis=0)              # psi_{t-1}
    bwd[0] *= -1.0
    ph = np.exp(1j * phi)
    diag_part = np.where(isA, fwd - ph * psi, psi - np.conj(ph) * bwd)
    return diag_part - delta * kappa * (psi @ h.T)


def apply_Mdag_brs(L, phi, psi, delta, kappa):
    """Adjoint of Eq. (2.2): (M^dag psi) = sum over rows of conj(M) psi.
    A sites: the forward difference transposes to psi_{x,t-1} (wrap sign at
    t = 0) and the diagonal to -e^{-i phi_{x,t}} psi_{x,t}; B sites: the
    diagonal 1 and the sub-diagonal of row t+1 (phase of time t+1) give
    psi_{x,t} - e^{+i phi_{x,t+1}} psi_{x,t+1} (wrap sign at t = Nt-1); the
    real symmetric hopping is its own adjoint."""
    Nt, V = phi.shape
    sub = lattice.sublattice(L)
    h = lattice.hopping_matrix(L)
    isA = (sub == 0)[None, :]
    bwd = np.roll(psi, 1, axis=0)              # psi_{t-1}
    bwd[0] *= -1.0
    fwd = np.roll(psi, -1, axis=0)             # psi_{t+1}
    fwd[Nt - 1] *= -1.0
    ph = np.exp(1j * phi)
    ph_next = np.roll(ph, -1, axis=0)          # e^{i phi_{t+1}}
    diag_part = np.where(isA, bwd - np.conj(ph) * psi, psi - ph_next * fwd)
    return diag_part - delta * kappa * (psi @ h.T)
