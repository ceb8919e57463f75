"""Krook-Wu exact solution of the homogeneous binary mixture (Sec. 6.1).

For the constant kernel B_ij = B_ji = lambda_ji / (4 pi n^(j)) the homogeneous equation
d_t f^(i) = sum_j Q^(ij)(f^(i), f^(j)) has the closed-form solution

    f^(i)(t, v) = n^(i) (m_i / (2 pi K))^(3/2) exp(-m_i v^2 / (2K)) ((1 - 3 Q_i) + m_i Q_i v^2 / K)

with mu, p_i, A, B, Q(t), Q_i = p_i Q, K(t) as defined in Sec. 6.1, and d_t f^(i) follows
by differentiating that expression (also printed there).  The paper's test takes
n^(1) = n^(2) = 1, lambda_11 = lambda_22 = 1, lambda_12 = lambda_21 = 1/2.
"""

import numpy as np


class KrookWu:
    def __init__(self, m1, m2, n=(1.0, 1.0), lam=((1.0, 0.5), (0.5, 1.0))):
        self.m = (float(m1), float(m2))
        self.n = (float(n[0]), float(n[1]))
        lam = np.asarray(lam, dtype=np.float64)
        self.lam = lam
        l11, l12, l21, l22 = lam[0, 0], lam[0, 1], lam[1, 0], lam[1, 1]
        mu = 4.0 * m1 * m2 / (m1 + m2) ** 2
        p1 = l22 - l21 * mu * (3.0 - 2.0 * mu)
        p2 = l11 - l12 * mu * (3.0 - 2.0 * mu)
        self.mu, self.p = mu, (p1, p2)
        self.A = (l11 + l21 * mu * (3.0 - 2.0 * mu * p2 / p1)) / 6.0
        self.B = (l11 * p1 + l21 * mu * (3.0 - 2.0 * mu) * p2) / 3.0
        # admissibility condition of the solution (Sec. 6.1)
        self.condition = (p1 - p2) * (2.0 * mu * mu * (l21 / p1 - l12 / p2) - 1.0)

    def kernel_prefactors(self):
        """b_ij = lambda_ji / (4 pi n^(j)) for the constant kernel (omega = 1, alpha = 1)."""
        b = np.zeros((2, 2))
        for i in range(2):
            for j in range(2):
                b[i, j] = self.lam[j, i] / (4.0 * np.pi * self.n[j])
        return b

    def Q(self, t):
        return self.A / (self.A * np.exp(self.A * t) - self.B)

    def dQ(self, t):
        e = np.exp(self.A * t)
        return -self.A ** 3 * e / (self.A * e - self.B) ** 2

    def K(self, t):
        n1, n2 = self.n
        p1, p2 = self.p
        return (n1 + n2) / ((n1 + n2) + 2.0 * (n1 * p1 + n2 * p2) * self.Q(t))

    def dK(self, t):
        n1, n2 = self.n
        p1, p2 = self.p
        den = (n1 + n2) + 2.0 * (n1 * p1 + n2 * p2) * self.Q(t)
        return -2.0 * (n1 + n2) * (n1 * p1 + n2 * p2) / den ** 2 * self.dQ(t)

    def f(self, i, t, v2):
        """f^(i)(t, v) for |v|^2 = v2 (any array shape)."""
        m, n = self.m[i], self.n[i]
        K = self.K(t)
        Qi = self.p[i] * self.Q(t)
        g = n * (m / (2.0 * np.pi * K)) ** 1.5 * np.exp(-m * v2 / (2.0 * K))
        return g * ((1.0 - 3.0 * Qi) + m / K * Qi * v2)

    def df(self, i, t, v2):
        """d_t f^(i)(t, v), the derivative formula of Sec. 6.1."""
        m, n = self.m[i], self.n[i]
        K, dK = self.K(t), self.dK(t)
        Qi, dQi = self.p[i] * self.Q(t), self.p[i] * self.dQ(t)
        g = n * (m / (2.0 * np.pi * K)) ** 1.5 * np.exp(-m * v2 / (2.0 * K))
        fi = self.f(i, t, v2)
        return (fi * (-1.5 / K * dK + m * v2 / (2.0 * K * K) * dK)
                + g * (-3.0 * dQi + m / K * dQi * v2 - m / (K * K) * dK * Qi * v2))
