"""The right-hand side of Eq. (cast) split into its terms, cell by cell, from the oracle's separately pinned
pieces (moments, Shakhov targets, J1, CD6, WENO-5 faces), for a periodic domain and chi_SET:

    L = (psi_S - psi) / tau + J1 - p (h_{i+1/2} - h_{i-1/2}) / dx.

Test infrastructure: used by tests only."""
import numpy as np

import oracle as O


def rhs_terms(m, phi, theta):
    """(relax_phi, relax_theta), (j1_phi, j1_theta), (adv_phi, adv_theta), each [nx][Q]."""
    p, w = O.velocity_set(m)
    nx, Q, dx = m.nx, m.Q, m.dx
    mom = np.array([O.moments(p, phi[i], theta[i]) for i in range(nx)])  # n, u, T, Pi, q
    n, u, T, q = mom[:, 0], mom[:, 1], mom[:, 2], mom[:, 4]
    lnn, lnT = np.log(n), np.log(T)

    def grad(f, i):
        return O.cd6(np.array([f[(i + r) % nx] for r in range(-3, 4)]), dx)

    relax = [np.zeros((nx, Q)), np.zeros((nx, Q))]
    j1 = [np.zeros((nx, Q)), np.zeros((nx, Q))]
    for i in range(nx):
        eta = m.eta0 * n[i] / m.rho_ref
        Y = 4.0 * eta * O.chi_set(eta)
        tau = O.tau(m, n[i], T[i])
        Pr = O.prandtl(m, n[i])
        dlnrho, du, dlnT = grad(lnn, i), grad(u, i), grad(lnT, i)
        dlnchi = eta * (3.0 / (1.0 - eta) - 1.0 / (2.0 - eta)) * dlnrho
        phS, thS = O.shakhov(p, w, n[i], u[i], T[i], q[i], Pr)
        relax[0][i] = (phS - phi[i]) / tau
        relax[1][i] = (thS - theta[i]) / tau
        if m.enskog:
            jp, jt = O.j1(p, w, n[i], u[i], T[i], Y, dlnchi, dlnrho, du, dlnT)
            j1[0][i], j1[1][i] = jp, jt
    adv = [np.zeros((nx, Q)), np.zeros((nx, Q))]
    for c, f in enumerate((phi, theta)):
        for k in range(Q):
            col = f[:, k]
            face = np.empty(nx)  # face[i]: interface i + 1/2
            for i in range(nx):
                if p[k] > 0:
                    s = [col[(i - 2 + r) % nx] for r in range(5)]
                else:
                    s = [col[(i + 3 - r) % nx] for r in range(5)]
                face[i] = O.weno5_face(np.array(s))
            adv[c][:, k] = p[k] * (face - np.roll(face, 1)) / dx
    return relax, j1, adv
